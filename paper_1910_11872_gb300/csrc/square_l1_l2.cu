// square_l1_l2.cu -- instantiations of the square-block solver for half-width(s) 1 2, both register-cap variants (square_variants.h).
#include "square_kernel.cuh"
#include "square_variants.h"

namespace rmusic {

RMUSIC_DEFINE_SQUARE(1)
RMUSIC_DEFINE_SQUARE(2)

}  // namespace rmusic
