// square_l8.cu -- instantiations of the square-block solver for half-width(s) 8, both register-cap variants (square_variants.h).
#include "square_kernel.cuh"
#include "square_variants.h"

namespace rmusic {

RMUSIC_DEFINE_SQUARE(8)

}  // namespace rmusic
