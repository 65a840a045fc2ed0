// sweep_r2.cu -- sweep variants of stencil radius 2 (space order 4).
#include "variants.h"
#include "wave_internal.h"

WAVE_DEFINE_RADIUS(2)
WAVE_DEFINE_MODES(2)
