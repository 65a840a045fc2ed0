// sweep_r6.cu -- sweep variants of stencil radius 6 (space order 12).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(6)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R6)
WAVE_DEFINE_MODES(6)
WAVE_DEFINE_TMULTI(6)
