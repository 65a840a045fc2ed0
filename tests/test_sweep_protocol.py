"""Randomised interleaving model of the sweep kernel's producer/consumer
mbarrier protocol (csrc/sweep.cuh): a producer warp fills ring U (level-n
planes, R+1+P deep) and ring K (level n-1 and coefficients, (T-1)R+1+P deep)
with TMA copies completed on per-iteration "full" barriers; consumers release
full phases through "consumed" barriers and ring slots through "empty"
barriers.  The first 2R iterations of a block load no ring-K data and stage s
reads only from iteration 2sR on.  The model checks,
over random schedules, that every slot a consumer reads holds the iteration
it expects, that no slot is overwritten while a consumer still reads it, that
the producer is never more than P+1 iterations ahead, and that the protocol
cannot deadlock.  It also checks that the model detects the hazard of a
protocol without the consumed barriers.

The untiled sweep (T = 1) runs without ring U (`split`): each ring-K slot
also takes the level-n plane of its own iteration for the x-queue (every
iteration) and the centre plane with halo (from iteration 2R on, with the
coefficients), and is released at the end of that iteration."""
import random


class MBar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0          # number of completed phases

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0, "too many arrivals in a phase"
        self._maybe_complete()

    def expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        assert self.tx >= 0
        self._maybe_complete()

    def _maybe_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait(self, parity):
        # true iff the phase with this parity has completed, i.e. current
        # (in-progress) phase parity != parity
        return (self.phase & 1) != parity


def simulate(R, T, P, niter, NT, seed, split=False):
    assert not split or T == 1
    rnd = random.Random(seed)
    DU, DK, DF = (0 if split else R + 1 + P), (T - 1) * R + 1 + P, P + 1
    full = [MBar(1) for _ in range(DF)]
    empF = [MBar(NT) for _ in range(DF)]
    empU = [MBar(NT) for _ in range(DU)]
    empK = [MBar(NT) for _ in range(DK)]
    total = niter
    slotU = [None] * DU   # iteration whose data is in the slot (None = garbage)
    slotK = [None] * DK
    slotF = [None] * DK   # split: iteration whose x-queue plane is in the slot
    inflight = []         # (iteration, U slot, K slot or None, full barrier)
    prod = dict(j=0, ju=0, jk=0, jf=0, ru=0, rk=0, rf=0, done=False)
    cons = [dict(g=0, su=0, sk=0, sf=0, pf=0, stage=0, done=False) for _ in range(NT)]
    waited = [[False] * total for _ in range(NT)]
    # the last iteration that reads a slot filled at iteration g
    last_u = lambda g: g + R                 # noqa: E731  (stage 1 centre plane)
    last_k = lambda g: g + (T - 1) * R       # noqa: E731  (stage T coefficients)
    steps = 0
    while True:
        steps += 1
        if steps > 400000:
            raise AssertionError("deadlock / livelock")
        actors = []
        if not prod["done"]:
            actors.append(("p", None))
        for i, c in enumerate(cons):
            if not c["done"]:
                actors.append(("c", i))
        if inflight:
            actors.append(("tma", None))
        if not actors:
            assert all(c["done"] for c in cons) and prod["done"], "deadlock"
            break
        kind, i = rnd.choice(actors)
        if kind == "tma":
            k = rnd.randrange(len(inflight))
            itr, dst_u, dst_k, bf, dst_f = inflight.pop(k)
            if dst_u is not None:
                slotU[dst_u] = itr
            if dst_k is not None:
                slotK[dst_k] = itr
            if dst_f is not None:
                slotF[dst_f] = itr
            full[bf].complete_tx(1)
        elif kind == "p":
            p = prod
            if p["j"] >= total:
                # drain: all issued loads complete before exit
                if inflight:
                    continue
                p["done"] = True
                continue
            j = p["j"]
            ok = True
            if p["rf"] > 0 and not empF[p["jf"]].try_wait((p["rf"] - 1) & 1):
                ok = False
            if ok and not split and p["ru"] > 0 and not empU[p["ju"]].try_wait((p["ru"] - 1) & 1):
                ok = False
            if ok and p["rk"] > 0 and not empK[p["jk"]].try_wait((p["rk"] - 1) & 1):
                ok = False
            if not ok:
                continue
            # invariant: slowest consumer has waited on iteration j - DF
            for ci in range(NT):
                if j - DF >= 0:
                    assert waited[ci][j - DF], "producer more than DF ahead"
            # the slots being overwritten must no longer be needed
            old_u = None if split else slotU[p["ju"]]
            if old_u is not None:
                for c in cons:
                    assert c["done"] or c["g"] > last_u(old_u), "U slot overwritten while needed"
            old_f = slotF[p["jk"]] if split else None
            if old_f is not None:
                for c in cons:
                    assert c["done"] or c["g"] > old_f, "queue-feed slot overwritten while needed"
            kload = j >= 2 * R
            old_k = slotK[p["jk"]]
            if kload and old_k is not None:
                for c in cons:
                    assert c["done"] or c["g"] > last_k(old_k), "K slot overwritten while needed"
            full[p["jf"]].expect_tx(1)
            if split:
                slotF[p["jk"]] = None
            else:
                slotU[p["ju"]] = None
            if kload:
                slotK[p["jk"]] = None
            inflight.append((j, None if split else p["ju"], p["jk"] if kload else None, p["jf"],
                             p["jk"] if split else None))
            if not split:
                p["ju"] += 1
                if p["ju"] == DU:
                    p["ju"] = 0
                    p["ru"] += 1
            p["jk"] += 1
            if p["jk"] == DK:
                p["jk"] = 0
                p["rk"] += 1
            p["jf"] += 1
            if p["jf"] == DF:
                p["jf"] = 0
                p["rf"] += 1
            p["j"] += 1
        else:
            c = cons[i]
            g = c["g"]
            if g >= total:
                c["done"] = True
                continue
            it = g
            if c["stage"] == 0:
                if not full[c["sf"]].try_wait(c["pf"]):
                    continue
                # level n of this iteration's plane (pushed into the queue)
                if split:
                    assert slotF[c["sk"]] == g, "stale queue-feed data"
                else:
                    assert slotU[c["su"]] == g, "stale U slot data"
                waited[i][g] = True
                empF[c["sf"]].arrive()
                c["stage"] = 1
                continue
            # stage s computes from local iteration 2sR on: stage 1 reads the
            # U slot of iteration g - R, stage s the K slot of g - (s-1)R
            for s in range(1, T + 1):
                if it < 2 * s * R:
                    continue
                if s == 1 and not split:
                    assert slotU[(c["su"] - R) % DU] == g - R, "U centre slot clobbered"
                jj = g - (s - 1) * R
                assert jj >= 2 * R
                assert slotK[(c["sk"] - (s - 1) * R) % DK] == jj, "K slot clobbered"
            if g >= R and not split:
                empU[(c["su"] - R) % DU].arrive()
            if g >= (T - 1) * R:
                empK[(c["sk"] - (T - 1) * R) % DK].arrive()
            c["stage"] = 0
            c["g"] += 1
            if not split:
                c["su"] = (c["su"] + 1) % DU
            c["sk"] = (c["sk"] + 1) % DK
            c["sf"] += 1
            if c["sf"] == DF:
                c["sf"] = 0
                c["pf"] ^= 1
    return steps


import pytest  # noqa: E402


@pytest.mark.parametrize("R", [1, 2, 4, 8])
@pytest.mark.parametrize("T", [1, 2, 3])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_protocol_random_schedules(R, T, P):
    for niter in (1, 3, 2 * R * T + 1, 2 * R * T + 5, 40):
        for seed in range(3):
            simulate(R, T, P, niter, 3, seed, split=False)
            if T == 1:
                simulate(R, T, P, niter, 3, seed, split=True)


_MUTATIONS = {
    # without the consumed barriers the producer can re-arm a full barrier
    # before every consumer waited on its previous phase (deep ring K, T >= 2)
    "no consumed barrier": [('if p["rf"] > 0 and not empF[p["jf"]].try_wait((p["rf"] - 1) & 1):',
                             "if False:")],
    # slots released before they were ever filled
    "release before the first fill": [("if g >= R and not split:", "if g >= 0 and not split:")],
    # a stage that starts before its x-queue holds the chunk's own planes
    "stage starts early": [("if it < 2 * s * R:", "if it < 2 * (s - 1) * R:")],
    # coefficient loads skipped for longer than the fill
    "ring K skipped too long": [("kload = j >= 2 * R", "kload = j >= 3 * R")],
    # a ring-K slot refilled without waiting for its release
    "no ring-K empty wait": [('if ok and p["rk"] > 0 and not empK[p["jk"]].try_wait((p["rk"] - 1) & 1):',
                              "if False:")],
}


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_model_detects_protocol_mistakes(name):
    import inspect
    src = inspect.getsource(simulate)
    for a, b in _MUTATIONS[name]:
        assert a in src
        src = src.replace(a, b)
    ns = dict(globals())
    exec(src, ns)
    caught = 0
    for R, T, P, split in [(1, 1, 1, False), (2, 2, 1, False), (4, 2, 2, False), (2, 3, 2, False),
                           (1, 1, 1, True), (4, 1, 2, True)]:
        for seed in range(3):
            try:
                ns["simulate"](R, T, P, 2 * R * T + 30, 3, seed, split=split)
            except AssertionError:
                caught += 1
    assert caught > 0
