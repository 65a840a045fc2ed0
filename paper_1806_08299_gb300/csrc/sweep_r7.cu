// sweep_r7.cu -- sweep variants of stencil radius 7 (space order 14).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(7)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R7)
WAVE_DEFINE_MODES(7)
WAVE_DEFINE_TMULTI(7)
