// sweep_r1.cu -- sweep variants of stencil radius 1 (space order 2).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(1)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R1)
WAVE_DEFINE_MODES(1)
WAVE_DEFINE_TMULTI(1)
