// k_source_tc.cu -- catastrophic-source angle contraction on the tensor cores
// (Remark 1, Section 4: sigma_c,s = sigma_c,t P^1 P^2; Appendix A.4):
//   src_g[a][yz] = du dv  sum_a'  P^2_g[a][a'] R_g[a'][yz]
// one dense GEMM per energy group, M = na (angles out), K = na (angles in),
// N = ny*nz (lateral points).  BF16 operands, FP32 accumulation, BF16 output.
//
// GB300 design (tcgen05, one CTA = 4 warps, 2 CTAs per SM):
//   * CTA tile M = 128 rows of P^2_g, N = 64 lateral points, the whole K = na;
//   * operands are staged by cp.async (16-byte chunks, zero-filled past the
//     ragged N edge) in the canonical no-swizzle layouts of the tensor core:
//     P^2 is K-major as it lies in memory ([a][a'], a' contiguous) and R is
//     MN-major as it lies in memory ([a'][yz], yz contiguous), so neither is
//     transposed;  8x8-element core matrices of 128 bytes, LBO = 128 B between
//     core matrices along K, SBO = (K/8) * 128 B between core matrices along M/N;
//   * one elected thread issues K/16 tcgen05.mma (kind::f16, BF16 x BF16 ->
//     FP32) into a 64-column TMEM accumulator and commits to an mbarrier;
//     the wait is bounded;
//   * the four warps read their 32 TMEM lanes (rows) with tcgen05.ld, scale by
//     du dv, convert to BF16 and store 128 contiguous bytes per row;
//   * each CTA walks a contiguous range of (g, M-tile, N-tile) tiles, so the
//     P^2 tile is reloaded only when (g, M-tile) changes.
#include "pbs_internal.cuh"

namespace pbs {

cudaError_t launch_source_bf16_cc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2,
                                  const __nv_bfloat16 *r, __nv_bfloat16 *src, double dudv, int nbatch);

namespace {

constexpr int kTM = 128;          // rows (out angles) per tile
constexpr int kTN = 64;           // lateral points per tile
constexpr int kThreads = 128;
constexpr int kTmemCols = 128;    // allocated (>= kTN, power of two)
constexpr long long kMmaWaitCycles = 4000000000LL;

__device__ __forceinline__ void cp_async_cg16(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory matrix descriptor (no swizzle): start, LBO, SBO in 16-byte
// units, fixed version bits 46..48 = 0b001, layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), A K-major (bit 15 = 0), B MN-major (bit 16 = 1),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads) k_source_tc(const __nv_bfloat16 *__restrict__ p2,
                                                         const __nv_bfloat16 *__restrict__ r,
                                                         __nv_bfloat16 *__restrict__ src, int na, int nyz, int ng,
                                                         int ngb, float dudv, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // [A tile: (kTM/8) * (na/8) * 128 B][B tile: (kTN/8) * (na/8) * 128 B]
  const int kcm = na / 8;  // core matrices along K
  unsigned char *sA = smem_raw;
  unsigned char *sB = smem_raw + (size_t)(kTM / 8) * kcm * 128;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  const int mtiles = na / kTM;
  const int ntiles = (nyz + kTN - 1) / kTN;
  const long long ntot = (long long)ngb * mtiles * ntiles;  // ngb = beams * ng (R, src blocks)
  const long long per = (ntot + gridDim.x - 1) / gridDim.x;
  const long long t_beg = blockIdx.x * per;
  const long long t_end = min(ntot, t_beg + per);
  const uint32_t idesc = idesc_bf16(kTM, kTN);
  const uint32_t lbo = 128, sbo = (uint32_t)kcm * 128;
  long long cur_a = -1;  // (g, M-tile) whose P^2 rows sit in sA
  unsigned phase = 0;

  for (long long t = t_beg; t < t_end; t++) {
    const int nt = (int)(t % ntiles);
    const long long gm = t / ntiles;  // g * mtiles + mt
    const int mt = (int)(gm % mtiles);
    const int gb = (int)(gm / mtiles);  // beam * ng + g
    const int g = gb % ng;
    const int n0 = nt * kTN;
    // ---- stage operands (cp.async, 16-byte chunks)
    if (gm != cur_a) {
      const __nv_bfloat16 *Ag = p2 + ((long long)g * na + (long long)mt * kTM) * na;
      // chunk (m, k8): rows m of the tile, 8 consecutive k
      for (int c = tid; c < kTM * kcm; c += kThreads) {
        const int m = c / kcm, kc = c % kcm;
        unsigned char *dst = sA + (size_t)(m >> 3) * kcm * 128 + (size_t)kc * 128 + (m & 7) * 16;
        cp_async_cg16(dst, Ag + (long long)m * na + kc * 8, 16u);
      }
      cur_a = gm;
    }
    {
      const __nv_bfloat16 *Bg = r + (long long)gb * na * nyz;
      // chunk (k, n8): row k of R_g, 8 consecutive lateral points
      for (int c = tid; c < na * (kTN / 8); c += kThreads) {
        const int k = c / (kTN / 8), nc = c % (kTN / 8);
        const int n = n0 + nc * 8;
        unsigned char *dst = sB + (size_t)nc * kcm * 128 + (size_t)(k >> 3) * 128 + (k & 7) * 16;
        const int valid = min(8, max(0, nyz - n));
        cp_async_cg16(dst, valid > 0 ? (const void *)(Bg + (long long)k * nyz + n) : (const void *)Bg,
                      (unsigned)(valid * 2));
      }
    }
    cp_async_wait_all();
    fence_proxy_async_smem();  // generic-proxy writes -> tensor-core (async proxy) reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- MMA: K/16 steps, one thread
    if (tid == 0) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int j = 0; j < na / 16; j++) {
        const uint64_t ad = smem_desc(a0 + (uint32_t)j * 256u, lbo, sbo);
        const uint64_t bd = smem_desc(b0 + (uint32_t)j * 256u, lbo, sbo);
        mma_bf16(tmem, ad, bd, idesc, j > 0);
      }
      mma_commit(&bar);
      if (!mbar_wait_bounded(&bar, phase, kMmaWaitCycles)) s_abort = 1;
    }
    phase ^= 1u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_abort) break;
    // ---- epilogue: warp w owns TMEM lanes (rows) 32w..32w+31
    {
      const int m = warp * 32 + lane;
      __nv_bfloat16 *out = src + ((long long)gb * na + (long long)mt * kTM + m) * nyz + n0;
#pragma unroll
      for (int half = 0; half < kTN / 32; half++) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * 32), v);
        const int nb = half * 32;
        if (n0 + nb + 32 <= nyz && (nyz % 8) == 0) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            uint4 pk;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v[q * 8 + 0] * dudv, v[q * 8 + 1] * dudv);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(v[q * 8 + 2] * dudv, v[q * 8 + 3] * dudv);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[q * 8 + 4] * dudv, v[q * 8 + 5] * dudv);
            __nv_bfloat162 h3 = __floats2bfloat162_rn(v[q * 8 + 6] * dudv, v[q * 8 + 7] * dudv);
            pk.x = *reinterpret_cast<uint32_t *>(&h0);
            pk.y = *reinterpret_cast<uint32_t *>(&h1);
            pk.z = *reinterpret_cast<uint32_t *>(&h2);
            pk.w = *reinterpret_cast<uint32_t *>(&h3);
            *reinterpret_cast<uint4 *>(out + nb + q * 8) = pk;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; i++)
            if (n0 + nb + i < nyz) out[nb + i] = __float2bfloat16_rn(v[i] * dudv);
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // TMEM reads done before the next tile's MMAs overwrite it
    tc_fence_after();
  }
  if (s_abort && tid == 0) {
    if (err) {
      atomicAdd(err, 1);
      atomicExch(err + 1, kErrTimeoutSourceMma);
    }
    // drain the outstanding MMA group (bounded) before TMEM is released
    mbar_wait_bounded(&bar, phase ^ 1u, kMmaWaitCycles / 8);
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

bool source_tc_supported(int na, int nyz) { return na % kTM == 0 && na <= 256 && nyz % 8 == 0; }

cudaError_t launch_source_tc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r,
                             __nv_bfloat16 *src, double dudv, int nbatch) {
  if (!source_tc_supported(d.na, d.nyz)) return launch_source_bf16_cc(lc, d, p2, r, src, dudv, nbatch);
  const size_t smem = (size_t)(kTM / 8 + kTN / 8) * (d.na / 8) * 128;
  cudaError_t e = cudaFuncSetAttribute(k_source_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_source_tc, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > 2) per_sm = 2;  // TMEM: 2 x 128 columns per SM
  const long long ntot = (long long)d.ng * nbatch * (d.na / kTM) * ((d.nyz + kTN - 1) / kTN);
  long long blocks = (long long)per_sm * lc.num_sms;
  if (blocks > ntot) blocks = ntot;
  k_source_tc<<<(unsigned)blocks, kThreads, smem, lc.stream>>>(p2, r, src, d.na, d.nyz, d.ng, d.ng * nbatch,
                                                               (float)dudv, lc.err);
  ++*lc.launches;
  return cudaGetLastError();
}

}  // namespace pbs
