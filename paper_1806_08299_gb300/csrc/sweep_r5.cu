// sweep_r5.cu -- sweep variants of stencil radius 5 (space order 10).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(5)
