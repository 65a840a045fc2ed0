// sweep_r4.cu -- sweep variants of stencil radius 4 (space order 8).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(4)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R4)
WAVE_DEFINE_MODES(4)
WAVE_DEFINE_TMULTI(4)
