// square_l3_l4.cu -- instantiations of the square-block solver for half-width(s) 3 4, both register-cap variants (square_variants.h).
#include "square_kernel.cuh"
#include "square_variants.h"

namespace rmusic {

RMUSIC_DEFINE_SQUARE(3)
RMUSIC_DEFINE_SQUARE(4)

}  // namespace rmusic
