// rmusic_validate.h -- validation of parameters and frame descriptors shared by every C entry point
// (the context-based entries in capi.cu and the allocation-free entry in noalloc.cu), so that the
// entries accept and reject the same inputs with the same codes.
#pragma once

#include "../../include/rmusic.h"
#include "rmusic_device.cuh"

namespace rmusic {

// RMUSIC_OK, or the code rmusic_create returns for these parameters (EINVAL for values outside
// their ranges or contradictory combinations, EUNSUPPORTED for valid ones no path implements).
int params_check(const rmusic_params& p);

// Frame-table entry of one descriptor under parameters p (which passed params_check): geometry of
// the carrier lines and window lines, kept band bins, work-item count. RMUSIC_OK, EINVAL for a
// malformed descriptor, EUNSUPPORTED for one the selected path does not handle.
int describe_frame(const rmusic_params& p, const rmusic_frame_desc& d, FrameDev* F);

}  // namespace rmusic
