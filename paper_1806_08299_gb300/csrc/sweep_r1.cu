// sweep_r1.cu -- sweep variants of stencil radius 1 (space order 2).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(1)
