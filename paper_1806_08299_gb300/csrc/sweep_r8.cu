// sweep_r8.cu -- sweep variants of stencil radius 8 (space order 16).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(8)
#define WAVE_MULTI_ARGS(...) WAVE_DEFINE_MULTI(__VA_ARGS__)
WAVE_MULTI_ARGS(WAVE_MULTI_R8)
WAVE_DEFINE_MODES(8)
WAVE_DEFINE_TMULTI(8)
