// sweep_r3.cu -- sweep variants of stencil radius 3 (space order 6).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(3)
