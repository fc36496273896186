// step_tma.h - launcher of the tensor-copy staged step kernel
// (lbm_step_tma.cu), for the C ABI's kernel dispatch.
#pragma once

#include "internal.h"

namespace lbm {

// 16-bit storage with the pulled values staged in shared memory by tensor
// copies: persistent over tiles whose shape `by` selects (1: 128 nodes x 2
// rows, 8: 64 x 8, any other value 64 x 4), periodic axes and halfway walls
// (not the on-site rule). err receives kErrTimeout if a bounded mbarrier
// wait gave up; cudaErrorNotSupported if the driver has no tensor-map
// encoder.
cudaError_t launch_step_tma(int storage, bool moments, const StepArgs &a, int *err, int by,
                            int sms, cudaStream_t s);

}  // namespace lbm
