// k_source_noalloc.cu -- allocation-free evaluation of the catastrophic source
// for callers that cannot allocate device memory themselves (for example code
// running inside an allocator-less host framework, or a process whose device
// memory is handed to it pre-carved by another owner).  Same arithmetic as
// pbs_eval_source on an FP32 context: the energy-summed source input R of
// one component, then src = du dv P^2_g R per group.  The only scratch, R, is
// a file-scope __device__ array; everything else is the caller's memory.
#include "pbs_internal.cuh"
#include "pbs.h"

#include <cmath>
#include <mutex>

namespace pbs {

namespace {

// Scratch for R: 4 Mi floats (16 MiB), held by every device that loads the
// library until the process exits.
constexpr long long kNoAllocMaxElems = 4LL << 20;
constexpr int kNoAllocMaxGroups = 2048;
__device__ __align__(256) float g_noalloc_r[kNoAllocMaxElems];

// Per-group coefficients of the exponential energy transfer, by value.
struct NoAllocCoef {
  float q1[kNoAllocMaxGroups];      // lambda sigma dE_g / Z_g
  float decay[kNoAllocMaxGroups];   // exp(-lambda (E_{g+1} - E_g)), 0 at the top
  float inv_de[kNoAllocMaxGroups];  // 1 / dE_g
};

// R_g = T_g / dE_g with T_g = rho q1_g psi^1_g + decay_g T_{g+1}, one thread per lane.
__global__ void k_source_input_noalloc(const float *__restrict__ psi, const float *__restrict__ rho_yz,
                                       float *__restrict__ r, int ng, long long lanes, int nyz,
                                       const __grid_constant__ NoAllocCoef cf) {
  const long long lane = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lane >= lanes) return;
  const float rho = rho_yz[lane % nyz];
  float t = 0.f;
  for (int g = ng - 1; g >= 0; g--) {
    t = rho * cf.q1[g] * psi[(long long)g * 2 * lanes + lane] + cf.decay[g] * t;
    r[(long long)g * lanes + lane] = t * cf.inv_de[g];
  }
}

std::mutex g_setup_mu;
float *g_scratch_ptr[64] = {};  // device address of g_noalloc_r per device ordinal

}  // namespace

}  // namespace pbs

using namespace pbs;

extern "C" pbs_status pbs_eval_source_noalloc(const float *psi_k, const float *rho_yz, const float *p2,
                                              const double *e_faces, int ng, int nu, int nv, int ny, int nz,
                                              double u_max, double v_max, double sigma_ct, double lambda_p1,
                                              float *src_out, void *stream) {
  if (!psi_k || !rho_yz || !p2 || !e_faces || !src_out) return PBS_ERR_ARG;
  if (ng < 1 || nu < 1 || nv < 1 || ny < 1 || nz < 1 || !(u_max > 0) || !(v_max > 0) || sigma_ct < 0 ||
      !(lambda_p1 > 0))
    return PBS_ERR_ARG;
  for (int f = 0; f < ng; f++)
    if (!(e_faces[f + 1] > e_faces[f])) return PBS_ERR_ARG;
  const long long na = (long long)nu * nv, nyz = (long long)ny * nz;
  if (ng > kNoAllocMaxGroups || (long long)ng * na * nyz > kNoAllocMaxElems) return PBS_ERR_UNSUPPORTED;

  // once per device, with that device current: the scratch array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PBS_ERR_CUDA;
  float *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_r) != cudaSuccess || !p) return PBS_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    scratch = g_scratch_ptr[dev];
  }

  // host FP64 coefficients of P^1 (exponential, normalised per emitting group)
  static NoAllocCoef cf;  // large: not on the stack; guarded by the mutex below
  std::lock_guard<std::mutex> lock(g_setup_mu);
  for (int gp = 0; gp < ng; gp++) {
    const double ecp = 0.5 * (e_faces[gp] + e_faces[gp + 1]);
    double z = 0.0;
    for (int g = 0; g <= gp; g++) z += lambda_p1 * std::exp(-lambda_p1 * (ecp - 0.5 * (e_faces[g] + e_faces[g + 1])));
    const double de = e_faces[gp + 1] - e_faces[gp];
    cf.q1[gp] = (float)(lambda_p1 * sigma_ct * de / z);
    cf.inv_de[gp] = (float)(1.0 / de);
    cf.decay[gp] = (gp + 1 < ng)
                       ? (float)std::exp(-lambda_p1 * (0.5 * (e_faces[gp + 1] + e_faces[gp + 2]) - ecp))
                       : 0.f;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long lanes = na * nyz;
  k_source_input_noalloc<<<(unsigned)((lanes + 255) / 256), 256, 0, st>>>(psi_k, rho_yz, scratch, ng, lanes,
                                                                          (int)nyz, cf);
  if (cudaGetLastError() != cudaSuccess) return PBS_ERR_CUDA;
  Dims d;
  d.ny = ny; d.nz = nz; d.ng = ng; d.nu = nu; d.nv = nv; d.na = (int)na; d.nyz = (int)nyz; d.ncomp = 1;
  d.nbeam = 1;
  d.lanes = lanes;
  d.comp_elems = (long long)ng * 2 * lanes;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PBS_ERR_CUDA;
  long long launches = 0;
  LaunchCtx lc{st, sms, &launches};
  const double du = 2.0 * u_max / (nu + 1), dv = 2.0 * v_max / (nv + 1);
  if (launch_source<float, float>(lc, d, p2, scratch, src_out, du * dv) != cudaSuccess) return PBS_ERR_CUDA;
  return PBS_OK;
}
