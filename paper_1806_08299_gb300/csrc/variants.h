// variants.h -- the sweep variants compiled into the library.
//
// X(R, T, BZ, BY, P): stencil radius R = space_order/2, time-tile depth T
// (T = 1: untiled sweep), output tile BZ (z) x BY (y) per block, TMA prefetch
// distance P planes.  Shared memory holds the TMA rings (2R+1+P level-n
// planes with halos; (T-1)R+1+P iterations of level n-1 and coefficients) and
// the centre planes of stages >= 2; registers hold (T-1)(2R+1)*4 floats of
// x-neighbour queues per thread.  Shapes are chosen so both fit an SM
// without spills (checked with -Xptxas -v).
#pragma once

#define WAVE_SWEEP_VARIANTS_R1(X) \
    X(1, 1, 64, 16, 2) X(1, 2, 64, 16, 2) X(1, 3, 64, 16, 2) X(1, 4, 56, 16, 2)
#define WAVE_SWEEP_VARIANTS_R2(X) \
    X(2, 1, 64, 16, 2) X(2, 1, 64, 8, 2) X(2, 2, 64, 16, 2) X(2, 3, 48, 12, 1) X(2, 4, 48, 8, 1)
#define WAVE_SWEEP_VARIANTS_R3(X) \
    X(3, 1, 64, 16, 2) X(3, 2, 56, 16, 1)
#define WAVE_SWEEP_VARIANTS_R4(X) \
    X(4, 1, 64, 16, 2) X(4, 1, 64, 8, 2) X(4, 2, 48, 16, 1) X(4, 2, 48, 8, 2)
#define WAVE_SWEEP_VARIANTS_R5(X) \
    X(5, 1, 64, 12, 2)
#define WAVE_SWEEP_VARIANTS_R6(X) \
    X(6, 1, 64, 12, 2)
#define WAVE_SWEEP_VARIANTS_R7(X) \
    X(7, 1, 64, 8, 2)
#define WAVE_SWEEP_VARIANTS_R8(X) \
    X(8, 1, 64, 8, 2)
