// sweep_r8.cu -- sweep variants of stencil radius 8 (space order 16).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(8)
