// k_source_tc.cu -- catastrophic-source angle contraction on the tensor cores.
#include "pbs_internal.cuh"

namespace pbs {

cudaError_t launch_source_bf16_cc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2,
                                  const __nv_bfloat16 *r, __nv_bfloat16 *src, double dudv);

cudaError_t launch_source_tc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r,
                             __nv_bfloat16 *src, double dudv) {
  return launch_source_bf16_cc(lc, d, p2, r, src, dudv);
}

}  // namespace pbs
