// variants.h -- the sweep variants compiled into the library.
//
// X(R, T, V, BZ, BY, P, MB): stencil radius R = space_order/2, time-tile depth T
// (T = 1: untiled sweep), V z-points per thread, output tile BZ (z) x BY (y)
// per block, TMA prefetch distance P planes, compiled for MB resident blocks
// per SM (the __launch_bounds__ minimum, which caps registers per thread).  Shared memory holds the TMA
// rings (T >= 2: R+1+P level-n planes with halos and (T-1)R+1+P iterations of
// level n-1 and coefficients; T = 1: 1+P iterations of the centre plane,
// the x-queue plane, level n-1 and coefficients) and the centre planes of
// stages >= 2; registers hold
// T (2R+1) V floats of x-neighbour queues per thread.  (T, BY, V, BZ) is
// unique per radius.  The first T = 1 entry of a radius is its default untiled
// variant (the fastest measured on GB300 where one was measured).
#pragma once

#define WAVE_SWEEP_VARIANTS_R1(X)                                                                  \
    X(1, 1, 2, 64, 8, 3, 3) X(1, 1, 4, 64, 16, 4, 2) X(1, 1, 8, 64, 16, 2, 2) X(1, 2, 4, 56, 16, 2, 2) \
    X(1, 3, 4, 56, 16, 2, 1) X(1, 4, 4, 56, 16, 2, 1) X(1, 4, 4, 56, 8, 1, 2)
#define WAVE_SWEEP_VARIANTS_R2(X)                                                                  \
    X(2, 1, 8, 64, 16, 2, 2) X(2, 1, 2, 64, 12, 2, 2) X(2, 1, 2, 64, 8, 3, 3) X(2, 1, 4, 64, 16, 4, 1) \
    X(2, 2, 4, 56, 16, 1, 1) X(2, 2, 2, 56, 16, 2, 1) X(2, 2, 4, 56, 8, 2, 2) X(2, 2, 4, 56, 12, 2, 2) \
    X(2, 2, 4, 120, 14, 1, 1) X(2, 2, 4, 120, 10, 2, 1) X(2, 2, 4, 128, 12, 1, 1) X(2, 3, 4, 56, 12, 2, 1) X(2, 4, 4, 48, 8, 1, 1)
#define WAVE_SWEEP_VARIANTS_R3(X) \
    X(3, 1, 2, 64, 12, 2, 2) X(3, 1, 4, 64, 16, 4, 1) X(3, 1, 8, 64, 16, 2, 2) X(3, 1, 4, 64, 12, 3, 2) \
    X(3, 2, 4, 56, 16, 1, 1)
#define WAVE_SWEEP_VARIANTS_R4(X)                                                                  \
    X(4, 1, 4, 64, 8, 2, 4) X(4, 1, 2, 64, 12, 2, 2) X(4, 1, 2, 64, 8, 3, 3) X(4, 1, 4, 64, 16, 4, 1) \
    X(4, 1, 8, 64, 12, 3, 2) X(4, 1, 8, 32, 24, 3, 2) X(4, 2, 4, 56, 16, 1, 1) X(4, 2, 2, 48, 16, 1, 1)     \
    X(4, 2, 4, 48, 8, 2, 1)
#define WAVE_SWEEP_VARIANTS_R5(X) \
    X(5, 1, 2, 64, 12, 2, 2) X(5, 1, 4, 64, 12, 3, 2) X(5, 1, 8, 64, 8, 3, 2) X(5, 1, 4, 64, 8, 3, 3)
#define WAVE_SWEEP_VARIANTS_R6(X) \
    X(6, 1, 2, 64, 8, 2, 2) X(6, 1, 4, 64, 12, 3, 2) X(6, 1, 8, 64, 8, 3, 2) X(6, 1, 4, 64, 8, 2, 3)
#define WAVE_SWEEP_VARIANTS_R7(X) \
    X(7, 1, 2, 64, 8, 2, 2) X(7, 1, 4, 64, 8, 2, 3) X(7, 1, 4, 64, 12, 2, 2)
#define WAVE_SWEEP_VARIANTS_R8(X) \
    X(8, 1, 2, 64, 8, 2, 2) X(8, 1, 4, 64, 8, 2, 3) X(8, 1, 4, 64, 12, 2, 2)

// Stage-specialised variants Z(R, T, V, VY, BZ, BY, P, MB) of tsweep.cuh:
// time step T on its own warps (T = 1 or 2), VY rows x V z-points per
// thread, output tile BZ x BY, TMA prefetch distance P, compiled for MB
// resident blocks per SM.  Shared memory holds P+1 slots of the stage-1
// inputs (centre box with halo, level n, level n-1, B, C over the stage-1
// region), for T = 2 also P+1 slots of the stage-2 inputs over the tile and
// R+3 planes of level n+1 handed from stage 1 to stage 2.  Registers hold a
// (2R+1)-plane x-queue of VY x V points per thread.  Each quarter of an SM
// has its own 16K registers and takes every fourth warp, so a block of w
// warps (times MB) can give a thread at most 16384 / (32 ceil(w MB / 4))
// registers: at so 16 (about 200 registers) no more than eight warps.
// MB = 0 is one block per SM of eight consumer warps and a producer
// warpgroup whose registers the consumers take over (setmaxnreg): eight
// consumer warps at up to 232 registers.
#define WAVE_TSWEEP_VARIANTS_R1(Z) Z(1, 1, 4, 1, 64, 8, 2, 3) Z(1, 2, 4, 2, 128, 12, 1, 1)
#define WAVE_TSWEEP_VARIANTS_R2(Z)                                                                 \
    Z(2, 1, 4, 1, 64, 8, 2, 2) Z(2, 1, 4, 2, 64, 16, 2, 2) Z(2, 2, 4, 2, 56, 24, 2, 1)            \
    Z(2, 2, 4, 2, 120, 12, 1, 1) Z(2, 2, 4, 2, 128, 12, 1, 1) Z(2, 2, 4, 2, 64, 24, 1, 1)           \
    Z(2, 2, 4, 1, 56, 16, 2, 1)
#define WAVE_TSWEEP_VARIANTS_R3(Z) Z(3, 1, 4, 2, 64, 16, 2, 2) Z(3, 2, 4, 2, 64, 24, 1, 1)
#define WAVE_TSWEEP_VARIANTS_R4(Z)                                                                 \
    Z(4, 1, 4, 1, 64, 8, 2, 2) Z(4, 1, 4, 2, 64, 16, 2, 2) Z(4, 2, 4, 2, 56, 24, 1, 1)             \
    Z(4, 2, 4, 2, 64, 24, 1, 1) Z(4, 2, 4, 2, 32, 32, 2, 1) Z(4, 2, 4, 2, 56, 16, 2, 1)            \
    Z(4, 2, 4, 1, 56, 16, 2, 1)
#define WAVE_TSWEEP_VARIANTS_R5(Z) Z(5, 1, 4, 2, 64, 16, 2, 2) Z(5, 2, 4, 2, 48, 16, 1, 1)
#define WAVE_TSWEEP_VARIANTS_R6(Z) \
    Z(6, 1, 4, 1, 64, 8, 2, 2) Z(6, 1, 4, 2, 64, 16, 2, 2) Z(6, 1, 4, 2, 64, 32, 2, 1) Z(6, 2, 4, 2, 32, 24, 1, 1)
#define WAVE_TSWEEP_VARIANTS_R7(Z) \
    Z(7, 1, 4, 2, 64, 16, 2, 1) Z(7, 1, 4, 2, 64, 32, 2, 0) Z(7, 1, 4, 2, 64, 32, 1, 0) Z(7, 2, 4, 2, 32, 16, 1, 0)
#define WAVE_TSWEEP_VARIANTS_R8(Z)                                                                 \
    Z(8, 1, 4, 1, 64, 8, 2, 2) Z(8, 1, 4, 2, 64, 16, 2, 1) Z(8, 1, 4, 2, 64, 24, 2, 1)             \
    Z(8, 2, 4, 2, 32, 8, 1, 1) Z(8, 1, 4, 2, 64, 32, 2, 0) Z(8, 1, 4, 2, 64, 32, 1, 0)             \
    Z(8, 1, 4, 2, 32, 64, 2, 0)

// Gradient-mode variants Y(R, T, V, BZ, BY, P, MB, XB): the untiled default
// shape of a radius with XB extra ring-K boxes (1: E for the second-difference
// sweep; 2: D and G for the imaging-condition sweep), so that those sweeps
// stream every input through TMA.  A shape without a mode variant runs its
// gradient sweeps on the plain variant, which reads the extras with ordinary
// loads.
#define WAVE_SWEEP_MODE_VARIANTS_R1(Y)
#define WAVE_SWEEP_MODE_VARIANTS_R2(Y) Y(2, 1, 8, 64, 16, 2, 2, 1) Y(2, 1, 8, 64, 16, 2, 2, 2)
#define WAVE_SWEEP_MODE_VARIANTS_R3(Y)
#define WAVE_SWEEP_MODE_VARIANTS_R4(Y) Y(4, 1, 4, 64, 8, 2, 3, 1) Y(4, 1, 4, 64, 8, 2, 3, 2)
#define WAVE_SWEEP_MODE_VARIANTS_R5(Y)
#define WAVE_SWEEP_MODE_VARIANTS_R6(Y)
#define WAVE_SWEEP_MODE_VARIANTS_R7(Y)
#define WAVE_SWEEP_MODE_VARIANTS_R8(Y)

// Gradient-mode variants of the stage-specialised sweep, Z(R, T, V, VY, BZ, BY,
// P, MB, MODE): MODE 1 (second differences stored; E streamed through TMA),
// MODE 2 (imaging condition; the D rows and G streamed through TMA).  A
// stage-specialised plan runs the mode variant of its own shape, or else the
// first of its depth (every shape gives the same bits); the extra boxes make
// the depth-2 slots larger, so so 8 has its own 32x32 shape.  MODE 3 (the
// Born perturbation sweep: D and the source coefficient streamed through
// TMA) has one untiled shape per radius, the only kernel that runs it.
// MODE 4 (the two-step Adams-Bashforth heat operator: the rate F in place of
// level n-1, handed to stage 2 beside level n+1) has untiled and depth-2
// shapes at so 2, 4 and 8 and an untiled one at so 16.  MODE 5 (the fused
// Born sweep: background and perturbation fields in one pass, two x-queues
// per thread) has one untiled shape per radius, one row per thread.
#define WAVE_TSWEEP_MODE_VARIANTS_R1(Z)                                                            \
    Z(1, 1, 4, 1, 64, 8, 2, 2, 3) Z(1, 1, 4, 1, 64, 8, 2, 2, 4) Z(1, 2, 4, 2, 128, 12, 1, 1, 4)      \
    Z(1, 1, 4, 1, 64, 8, 2, 2, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R2(Z)                                                            \
    Z(2, 1, 4, 1, 64, 8, 2, 2, 1) Z(2, 1, 4, 1, 64, 8, 2, 2, 2) Z(2, 2, 4, 2, 128, 12, 1, 1, 1)    \
    Z(2, 2, 4, 2, 128, 12, 1, 1, 2) Z(2, 1, 4, 1, 64, 8, 2, 2, 3) Z(2, 1, 4, 1, 64, 8, 2, 2, 4)      \
    Z(2, 2, 4, 2, 128, 12, 1, 1, 4) Z(2, 1, 4, 1, 64, 8, 2, 2, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R3(Z) Z(3, 1, 4, 2, 64, 16, 2, 2, 3) Z(3, 1, 4, 1, 64, 8, 2, 2, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R4(Z)                                                            \
    Z(4, 1, 4, 2, 64, 16, 2, 2, 1) Z(4, 1, 4, 2, 64, 16, 2, 2, 2) Z(4, 2, 4, 2, 32, 32, 1, 1, 1)   \
    Z(4, 2, 4, 2, 32, 32, 1, 1, 2) Z(4, 1, 4, 2, 64, 16, 2, 2, 3) Z(4, 1, 4, 2, 64, 16, 2, 2, 4)    \
    Z(4, 2, 4, 2, 56, 16, 2, 1, 4) Z(4, 1, 4, 1, 64, 8, 2, 2, 5) Z(4, 2, 4, 1, 32, 24, 1, 1, 1)    \
    Z(4, 2, 4, 1, 32, 24, 1, 1, 2) Z(4, 1, 4, 1, 64, 8, 2, 3, 1) Z(4, 1, 4, 1, 64, 8, 2, 3, 2)
#define WAVE_TSWEEP_MODE_VARIANTS_R5(Z) Z(5, 1, 4, 2, 64, 16, 2, 2, 3) Z(5, 1, 4, 1, 64, 8, 2, 2, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R6(Z) Z(6, 1, 4, 2, 64, 16, 2, 2, 3) Z(6, 1, 4, 1, 64, 8, 2, 1, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R7(Z) Z(7, 1, 4, 2, 64, 32, 2, 0, 3) Z(7, 1, 4, 1, 64, 8, 2, 1, 5)
#define WAVE_TSWEEP_MODE_VARIANTS_R8(Z) Z(8, 1, 4, 2, 64, 32, 2, 0, 3) Z(8, 1, 4, 2, 64, 32, 2, 0, 4)  \
    Z(8, 1, 4, 1, 64, 8, 2, 1, 5)

// Batched stage-specialised variants M(R, T, V, VY, BZ, BY, P, MB, MODE): the
// sweeps of a survey group on the stage-specialised kernel, each the batched
// form of the single-shot variant of the same shape and mode (0 forward, 1
// the gradient's recompute, 2 its imaging-condition adjoint).
#define WAVE_TMULTI_VARIANTS_R1(M)
#define WAVE_TMULTI_VARIANTS_R2(M)                                                                 \
    M(2, 1, 4, 1, 64, 8, 2, 2, 0) M(2, 2, 4, 2, 128, 12, 1, 1, 0) M(2, 1, 4, 1, 64, 8, 2, 2, 1)      \
    M(2, 1, 4, 1, 64, 8, 2, 2, 2) M(2, 2, 4, 2, 128, 12, 1, 1, 1) M(2, 2, 4, 2, 128, 12, 1, 1, 2)
#define WAVE_TMULTI_VARIANTS_R3(M)
#define WAVE_TMULTI_VARIANTS_R4(M)                                                                 \
    M(4, 1, 4, 2, 64, 16, 2, 2, 0) M(4, 2, 4, 2, 64, 24, 1, 1, 0) M(4, 1, 4, 2, 64, 16, 2, 2, 1)     \
    M(4, 1, 4, 2, 64, 16, 2, 2, 2) M(4, 2, 4, 2, 32, 32, 1, 1, 1) M(4, 2, 4, 2, 32, 32, 1, 1, 2)
#define WAVE_TMULTI_VARIANTS_R5(M)
#define WAVE_TMULTI_VARIANTS_R6(M)
#define WAVE_TMULTI_VARIANTS_R7(M)
#define WAVE_TMULTI_VARIANTS_R8(M)

// Batched-kernel shape per radius (its default untiled shape): all shots of a
// batch advance in one launch per time step.
#define WAVE_MULTI_R1 1, 1, 2, 64, 8, 3, 3
#define WAVE_MULTI_R2 2, 1, 8, 64, 16, 2, 2
#define WAVE_MULTI_R3 3, 1, 2, 64, 12, 2, 2
#define WAVE_MULTI_R4 4, 1, 4, 64, 8, 2, 4
#define WAVE_MULTI_R5 5, 1, 2, 64, 12, 2, 2
#define WAVE_MULTI_R6 6, 1, 2, 64, 8, 2, 2
#define WAVE_MULTI_R7 7, 1, 2, 64, 8, 2, 2
#define WAVE_MULTI_R8 8, 1, 2, 64, 8, 2, 2
