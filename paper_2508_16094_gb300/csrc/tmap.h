// The driver's tensor-map encoder, resolved once at run time (the library does
// not link libcuda's symbols directly).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

namespace gipm {

// cuTensorMapEncodeTiled; throws std::runtime_error when the driver lacks it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace gipm
