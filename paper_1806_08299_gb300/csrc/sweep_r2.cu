// sweep_r2.cu -- sweep variants of stencil radius 2 (space order 4).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(2)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R2)
WAVE_DEFINE_MODES(2)
WAVE_DEFINE_TMULTI(2)
