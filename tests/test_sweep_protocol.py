"""Randomised interleaving model of the sweep kernel's producer/consumer
mbarrier protocol (csrc/sweep.cuh): a producer warp fills ring U (level-n
planes, R+1+P deep) and ring K (level n-1 and coefficients, (T-1)R+1+P deep)
with TMA copies completed on per-iteration "full" barriers; consumers release
full phases through "consumed" barriers and ring slots through "empty"
barriers.  The model checks, over random schedules, that no slot is
overwritten while a consumer still reads it, that consumers never see a
skipped phase, that the producer is never more than P+1 iterations ahead, and
that the protocol cannot deadlock.  It also checks that the model detects the
hazard of a protocol without the consumed barriers."""
import random
import sys


class MBar:
    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0          # number of completed phases
        self.armed_tx = False

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


def simulate(R, T, P, niter, NT, seed):
    rnd = random.Random(seed)
    DU, DK, DF = R + 1 + P, (T - 1) * R + 1 + P, P + 1
    full = [MBar(1) for _ in range(DF)]
    empF = [MBar(NT) for _ in range(DF)]
    empU = [MBar(NT) for _ in range(DU)]
    empK = [MBar(NT) for _ in range(DK)]
    slotU = [None] * DU   # iteration whose data is in the slot (None = garbage)
    slotK = [None] * DK
    inflight = []         # (iteration, remaining steps)
    # producer state
    prod = dict(j=0, ju=0, jk=0, jf=0, ru=0, rk=0, rf=0, stage=0, done=False)
    cons = [dict(it=0, su=0, sk=0, sf=0, pf=0, stage=0, done=False) for _ in range(NT)]
    waited = [[False] * niter for _ in range(NT)]
    steps = 0
    while True:
        steps += 1
        if steps > 200000:
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
            break
        kind, i = rnd.choice(actors)
        if kind == "tma":
            k = rnd.randrange(len(inflight))
            itr, dst_u, dst_k, bf = inflight.pop(k)
            slotU[dst_u] = itr
            slotK[dst_k] = itr
            full[bf].complete_tx(1)
        elif kind == "p":
            p = prod
            if p["j"] >= niter:
                # drain: all issued loads complete before exit
                if inflight:
                    continue
                p["done"] = True
                continue
            j = p["j"]
            ok = True
            if p["rf"] > 0 and not empF[p["jf"]].try_wait((p["rf"] - 1) & 1):
                ok = False
            if ok and p["ru"] > 0 and not empU[p["ju"]].try_wait((p["ru"] - 1) & 1):
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
            old_u = slotU[p["ju"]]
            if old_u is not None:
                for c in cons:
                    assert c["done"] or c["it"] > old_u + R, "U slot overwritten while needed"
            old_k = slotK[p["jk"]]
            if old_k is not None:
                for c in cons:
                    assert c["done"] or c["it"] > old_k + (T - 1) * R, "K slot overwritten while needed"
            full[p["jf"]].expect_tx(1)
            slotU[p["ju"]] = None
            slotK[p["jk"]] = None
            inflight.append((j, p["ju"], p["jk"], p["jf"]))
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
            it = c["it"]
            if it >= niter:
                c["done"] = True
                continue
            if c["stage"] == 0:
                if not full[c["sf"]].try_wait(c["pf"]):
                    continue
                # data of iteration it must be present
                assert slotU[c["su"]] == it and slotK[c["sk"]] == it, "stale slot data"
                waited[i][it] = True
                empF[c["sf"]].arrive()
                c["stage"] = 1
                continue
            # compute: reads U slot of it - R and K slots of it .. it - (T-1)R
            if it - R >= 0:
                su = (c["su"] - R) % DU
                assert slotU[su] == it - R, "U centre slot clobbered"
            for s in range(1, T + 1):
                jj = it - (s - 1) * R
                if jj >= 0:
                    assert slotK[(c["sk"] - (s - 1) * R) % DK] == jj, "K slot clobbered"
            if it >= R:
                empU[(c["su"] - R) % DU].arrive()
            if it >= (T - 1) * R:
                empK[(c["sk"] - (T - 1) * R) % DK].arrive()
            c["stage"] = 0
            c["it"] += 1
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
    for niter in (1, 3, 2 * R * T + 5, 40):
        for seed in range(3):
            simulate(R, T, P, niter, 3, seed)


def test_model_detects_missing_consumed_barrier():
    # without the consumed barriers the producer can re-arm a full barrier
    # before every consumer waited on its previous phase (deep ring K, T >= 2)
    import inspect
    src = inspect.getsource(simulate).replace(
        'if p["rf"] > 0 and not empF[p["jf"]].try_wait((p["rf"] - 1) & 1):', "if False:")
    ns = dict(globals())
    exec(src, ns)
    caught = 0
    for seed in range(20):
        try:
            ns["simulate"](4, 2, 2, 40, 3, seed)
        except AssertionError:
            caught += 1
    assert caught > 0
