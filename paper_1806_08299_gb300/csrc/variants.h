// variants.h -- the sweep variants compiled into the library.
//
// X(R, T, V, BZ, BY): stencil radius R = space_order/2, time-tile depth T
// (T = 1: untiled sweep), V z-points per thread, output tile BZ x BY.
// Sizes are chosen so that the register queues (T * (2R+1) * V floats per
// thread) of one block fit one SM's register file without spills
// (checked with -Xptxas -v).
#pragma once

#define WAVE_SWEEP_VARIANTS_R1(X) \
    X(1, 1, 4, 64, 16) X(1, 2, 4, 64, 16) X(1, 3, 4, 64, 16) X(1, 4, 4, 56, 16)
#define WAVE_SWEEP_VARIANTS_R2(X) \
    X(2, 1, 4, 64, 16) X(2, 2, 4, 64, 16) X(2, 3, 4, 48, 16) X(2, 4, 4, 48, 12)
#define WAVE_SWEEP_VARIANTS_R3(X) \
    X(3, 1, 4, 64, 16) X(3, 2, 4, 56, 16)
#define WAVE_SWEEP_VARIANTS_R4(X) \
    X(4, 1, 4, 64, 16) X(4, 2, 4, 48, 16)
#define WAVE_SWEEP_VARIANTS_R5(X) \
    X(5, 1, 4, 64, 12)
#define WAVE_SWEEP_VARIANTS_R6(X) \
    X(6, 1, 4, 64, 12)
#define WAVE_SWEEP_VARIANTS_R7(X) \
    X(7, 1, 4, 64, 8)
#define WAVE_SWEEP_VARIANTS_R8(X) \
    X(8, 1, 4, 64, 8)
