// oz_slicegemm on the 5th-generation tensor cores (tcgen05): placeholder
// until the kernel lands; the mma.sync kernel serves meanwhile.
#include "common.cuh"
#include "kernels.h"

namespace mpc {

cudaError_t launch_slicegemm_tc(const SliceGemmArgs &, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace mpc
