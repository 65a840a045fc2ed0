// sweep_r6.cu -- sweep variants of stencil radius 6 (space order 12).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(6)
