// sweep_r3.cu -- sweep variants of stencil radius 3 (space order 6).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(3)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R3)
WAVE_DEFINE_MODES(3)
WAVE_DEFINE_TMULTI(3)
