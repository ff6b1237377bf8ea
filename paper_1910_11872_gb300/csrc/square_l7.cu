// square_l7.cu -- instantiations of the square-block solver for half-width(s) 7, both register-cap variants (square_variants.h).
#include "square_kernel.cuh"
#include "square_variants.h"

namespace rmusic {

RMUSIC_DEFINE_SQUARE(7)

}  // namespace rmusic
