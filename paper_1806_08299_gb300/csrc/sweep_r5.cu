// sweep_r5.cu -- sweep variants of stencil radius 5 (space order 10).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(5)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R5)
WAVE_DEFINE_MODES(5)
WAVE_DEFINE_TMULTI(5)
