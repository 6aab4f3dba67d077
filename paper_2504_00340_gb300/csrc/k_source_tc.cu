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

// The same with the 128-byte swizzle (layout type 2, bits 61..63): rows of
// 128 bytes, XOR-swizzled in 1024-byte atoms of 8 rows; start addresses on
// atom boundaries (base offset 0).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
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

// The NK MMAs (K = 16 each) of one accumulator tile: the first overwrites D,
// the others accumulate.  A descriptor's start address (16-byte units, bits
// 0-13; shared addresses stay below 2^18 bytes, so the field never carries
// into the rest of the low word) steps by 256 bytes along K for A and by
// BSTEP 16-byte units for B: one 32-bit add per descriptor per MMA.
__device__ __forceinline__ void mma_bf16_w(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
      "mov.b64 da, {%1, %2};\n\t"
      "mov.b64 db, {%3, %4};\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}" ::"r"(tmem_d),
      "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(accumulate)
      : "memory");
}
template <int NK, uint32_t BSTEP>
__device__ __forceinline__ void mma_chain(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc) {
  const uint32_t alo = (uint32_t)ad, ahi = (uint32_t)(ad >> 32), blo = (uint32_t)bd, bhi = (uint32_t)(bd >> 32);
#pragma unroll
  for (int j = 0; j < NK; j++) mma_bf16_w(d, alo + 16u * j, ahi, blo + BSTEP * j, bhi, idesc, j > 0 ? 1u : 0u);
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

// 256-bit global store of eight 32-bit words (32-byte aligned address).
__device__ __forceinline__ void st_global_v8(void *p, const uint32_t *w) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
               "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
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

// ---------------------------------------------------------------- pipelined form
//
// Warp-specialised and pipelined: lane 0 of warp 0 issues the TMA loads, lane
// 0 of warp 1 the MMAs, warps 2-9 drain the accumulators.  P^2_g (all M rows,
// whole K) is loaded once per group by one 5-D TMA copy straight into the canonical K-major
// core-matrix layout; each R tile (whole K x 64 lateral points) by one 3-D TMA
// copy into the canonical MN-major layout, kPipeMax stages ahead; the MMAs of a
// tile go into one of four TMEM accumulators while the epilogue warps drain
// the others, so loads, MMAs and stores of consecutive tiles overlap and the
// MMAs run up to three tiles ahead of the stores.  Two epilogue warps share
// each TMEM lane quadrant, one per 32-column half of the tile; each thread
// writes its row's 32 BF16 values as two whole 32-byte sectors.  The MMAs of a
// tile are issued from descriptors stepped by one 32-bit add each (the start
// address field moves along K), so the issuing thread keeps the tensor pipe
// fed; the loads wait only for free stages and, at a group change, for the
// MMAs that read the old P^2 (an MMA commit releases it).
// Each CTA walks a contiguous range of (group, N-tile) tiles; every wait is
// bounded.

constexpr int kPipeMax = 4;                      // R stages (3 when na = 256: shared memory)
constexpr int kPipeThreads = 320;                // warp 0: TMA producer; warp 1: MMA issue; warps 2-9: epilogue
constexpr int kEpiThreads = kPipeThreads - 64;
constexpr int kAcc = 4;                          // TMEM accumulators (4 x 128 columns when na = 256)
constexpr long long kPipeWait = 2000000000LL;    // ~1 s at 2 GHz

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// SWB: the R tile arrives as [k][64 lateral points] rows of 128 bytes with the
// 128-byte swizzle (one TMA row per k, instead of 8 segments of 16 bytes),
// described as MN-major with 8-row groups 1024 bytes apart along K.
template <bool SWB>
__global__ void __launch_bounds__(kPipeThreads, 1)
    k_source_tc_pipe(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     __nv_bfloat16 *__restrict__ src, int na, int nyz, int ng, int ngb, int nstages, float dudv,
                     int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int mh = na / kTM;  // M halves
  const int kcm = na / 8;
  const unsigned a_bytes = (unsigned)na * na * 2u;
  const unsigned b_bytes = (unsigned)na * kTN * 2u;
  unsigned char *sA = smem_raw;
  unsigned char *sB = smem_raw + a_bytes;  // stage s at sB + s * b_bytes
  __shared__ __align__(8) uint64_t full_b[kPipeMax], empty_b[kPipeMax], acc_full[kAcc], acc_empty[kAcc], a_full, a_empty;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int acc_cols = mh * kTN;  // columns of one accumulator (both M halves)
  const uint32_t tmem_cols = (uint32_t)(kAcc * acc_cols);  // 512 (na = 256) or 256 (na = 128)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kPipeMax; i++) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
    }
    for (int i = 0; i < kAcc; i++) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kEpiThreads);
    }
    mbar_init(&a_full, 1);
    mbar_init(&a_empty, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  const int ntn = (nyz + kTN - 1) / kTN;
  const long long ntot = (long long)ngb * ntn;
  const long long per = (ntot + gridDim.x - 1) / gridDim.x;
  const long long t_beg = (long long)blockIdx.x * per;
  const long long t_end = min(ntot, t_beg + per);
  const int count = (int)max(0LL, t_end - t_beg);

  if (warp == 0) {
    if (lane == 0 && count > 0) {
      // TMA producer: R tiles nstages ahead; P^2 of a new group once the MMAs
      // reading the old one have completed (a_empty, committed by the MMA lane)
      int issued = 0, cur_gb = -1, n_a = 0;
      bool ok = true, a_pending = false;
      for (; issued < count && ok; issued++) {
        if (*reinterpret_cast<volatile int *>(&s_abort)) break;
        const int s = issued % nstages;
        if (issued >= nstages) ok = mbar_wait_bounded(&empty_b[s], (unsigned)((issued / nstages - 1) & 1), kPipeWait);
        if (!ok) break;
        const long long t = t_beg + issued;
        const int gb = (int)(t / ntn), nt = (int)(t % ntn);
        mbar_arrive_expect_tx(&full_b[s], b_bytes);
        if (SWB)
          tma_load_2d(sB + (size_t)s * b_bytes, &mapB, nt * kTN, gb * na, &full_b[s]);
        else
          tma_load_3d(sB + (size_t)s * b_bytes, &mapB, 0, gb * na, nt * (kTN / 8), &full_b[s]);
        if (gb != cur_gb) {
          if (n_a > 0) ok = mbar_wait_bounded(&a_empty, (unsigned)((n_a - 1) & 1), kPipeWait);
          if (!ok) {
            issued++;  // this tile's R copy is in flight
            break;
          }
          mbar_arrive_expect_tx(&a_full, a_bytes);
          tma_load_5d(sA, &mapA, 0, 0, 0, 0, gb % ng, &a_full);
          a_pending = true;
          n_a++;
          cur_gb = gb;
        }
      }
      if (!ok) {
        *reinterpret_cast<volatile int *>(&s_abort) = 1;
        if (err) {
          atomicAdd(err, 1);
          atomicExch(err + 1, kErrTimeoutSourceMma);
        }
      }
      // every copy this lane issued lands before the CTA exits (bounded): the
      // last copy into each stage, and the last P^2 copy
      for (int k = (issued > nstages ? issued - nstages : 0); k < issued; k++)
        mbar_wait_bounded(&full_b[k % nstages], (unsigned)((k / nstages) & 1), kPipeWait / 8);
      if (a_pending) mbar_wait_bounded(&a_full, (unsigned)((n_a - 1) & 1), kPipeWait / 8);
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0) {
      // MMA issue: one accumulator tile per R tile, four accumulators in turn
      const uint32_t idesc = idesc_bf16(kTM, kTN);
      const uint32_t lbo = 128, sbo = (uint32_t)kcm * 128;
      const uint64_t adesc = smem_desc(smem_u32(sA), lbo, sbo);
      int cur_gb = -1, n_a = 0, committed = 0;
      bool ok = true;
      for (int i = 0; i < count && ok; i++) {
        const long long t = t_beg + i;
        const int gb = (int)(t / ntn);
        if (gb != cur_gb) {
          // release the old P^2 (completes when every MMA issued so far has),
          // then wait for the new one
          if (n_a > 0) mma_commit(&a_empty);
          ok = mbar_wait_bounded(&a_full, (unsigned)(n_a & 1), kPipeWait);
          if (!ok) break;
          n_a++;
          cur_gb = gb;
        }
        const int s = i % nstages;
        ok = mbar_wait_bounded(&full_b[s], (unsigned)((i / nstages) & 1), kPipeWait);
        if (!ok) break;
        const int acc = i % kAcc;
        if (i >= kAcc) ok = mbar_wait_bounded(&acc_empty[acc], (unsigned)((i / kAcc - 1) & 1), kPipeWait);
        if (!ok) break;
        if (*reinterpret_cast<volatile int *>(&s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // K = 16 per MMA: two 8-row groups of the B tile (2 x 1024 B swizzled,
        // or 2 core matrices of 128 B) and 2 core matrices of A
        const uint32_t b0 = smem_u32(sB + (size_t)s * b_bytes);
        const uint64_t bd0 = SWB ? smem_desc_sw128(b0, 0u, 1024u) : smem_desc(b0, lbo, sbo);
        for (int h = 0; h < mh; h++) {
          const uint64_t ad0 = adesc + (uint64_t)(((uint32_t)h * (kTM / 8) * kcm * 128u) >> 4);
          const uint32_t d = tmem + (uint32_t)(acc * acc_cols + h * kTN);
          if (na == 256)
            mma_chain<16, SWB ? 128u : 16u>(d, ad0, bd0, idesc);
          else
            mma_chain<8, SWB ? 128u : 16u>(d, ad0, bd0, idesc);
        }
        mma_commit(&empty_b[s]);
        mma_commit(&acc_full[acc]);
        committed = i + 1;
      }
      if (!ok) {
        *reinterpret_cast<volatile int *>(&s_abort) = 1;
        if (err) {
          atomicAdd(err, 1);
          atomicExch(err + 1, kErrTimeoutSourceMma);
        }
      }
      // the last commit covers every MMA issued (tile committed - 1; fewer than
      // count after a timeout): wait for it before TMEM is released
      if (committed > 0)
        mbar_wait_bounded(&acc_full[(committed - 1) % kAcc], (unsigned)(((committed - 1) / kAcc) & 1), kPipeWait);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 of each M half,
    // columns 32 half .. +31 of the tile (half = (w - 2) / 4)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    // BF16 rows of a multiple of 32 bytes from a 32-byte aligned base
    const bool sector_rows = (nyz & 15) == 0 && (reinterpret_cast<uintptr_t>(src) & 31) == 0;
    for (int i = 0; i < count; i++) {
      const int acc = i % kAcc;
      const bool ok = mbar_wait_bounded(&acc_full[acc], (unsigned)((i / kAcc) & 1), kPipeWait);
      // warp-uniform decision: the TMEM loads below are warp-collective
      if (!__all_sync(0xffffffffu, ok && *reinterpret_cast<volatile int *>(&s_abort) == 0)) break;
      tc_fence_after();
      const long long t = t_beg + i;
      const int gb = (int)(t / ntn);
      const int n1 = (int)(t % ntn) * kTN + half * 32;  // first lateral point of this warp's columns
      for (int h = 0; h < mh; h++) {
        const int m = h * kTM + q * 32 + lane;
        __nv_bfloat16 *out = src + ((long long)gb * na + m) * nyz + n1;
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * acc_cols + h * kTN + half * 32), v);
        if (n1 + 32 <= nyz) {
          uint32_t w[16];
#pragma unroll
          for (int c = 0; c < 16; c++) {
            __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * c] * dudv, v[2 * c + 1] * dudv);
            w[c] = *reinterpret_cast<uint32_t *>(&b);
          }
          if (sector_rows) {
            st_global_v8(out, w);
            st_global_v8(out + 16, w + 8);
          } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
              *reinterpret_cast<uint4 *>(out + c * 8) = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 32; e++)
            if (n1 + e < nyz) out[e] = __float2bfloat16_rn(v[e] * dudv);
        }
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[acc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Tensor maps of the pipelined form: P^2 as [g][m8][kc][m7][k8] (5-D box = one
// group) and R as [chunk][row][n8] (3-D box = whole K x 64 lateral points) or,
// swizzled, as [row][64 n] (2-D box, 128-byte swizzle).
bool source_pipe_maps(const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r, int nbatch, bool swb,
                      CUtensorMap &ma, CUtensorMap &mb) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t na = (cuuint64_t)d.na, nyz = (cuuint64_t)d.nyz;
  {
    cuuint64_t dims[5] = {8, 8, na / 8, na / 8, (cuuint64_t)d.ng};
    cuuint64_t strides[4] = {na * 2, 16, 8 * na * 2, na * na * 2};
    cuuint32_t box[5] = {8, 8, (cuuint32_t)(na / 8), (cuuint32_t)(na / 8), 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(p2), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (swb) {
    cuuint64_t dims[2] = {nyz, (cuuint64_t)d.ng * nbatch * na};
    cuuint64_t strides[1] = {nyz * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTN, (cuuint32_t)na};
    cuuint32_t es[2] = {1, 1};
    if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(r), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  } else {
    cuuint64_t dims[3] = {8, (cuuint64_t)d.ng * nbatch * na, nyz / 8};
    cuuint64_t strides[2] = {nyz * 2, 16};
    cuuint32_t box[3] = {8, (cuuint32_t)na, kTN / 8};
    cuuint32_t es[3] = {1, 1, 1};
    if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(r), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace

bool source_tc_supported(int na, int nyz) { return na % kTM == 0 && na <= 256 && nyz % 8 == 0; }

cudaError_t launch_source_tc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r,
                             __nv_bfloat16 *src, double dudv, int nbatch) {
  if (!source_tc_supported(d.na, d.nyz)) return launch_source_bf16_cc(lc, d, p2, r, src, dudv, nbatch);
  CUtensorMap ma, mb;
  const bool swb = lc.source_form == 2;
  if (lc.source_form >= 1 && source_pipe_maps(d, p2, r, nbatch, swb, ma, mb)) {
    const int nstages = d.na == 256 ? 3 : kPipeMax;
    const size_t smem = (size_t)d.na * d.na * 2 + (size_t)nstages * d.na * kTN * 2;
    auto kern = swb ? k_source_tc_pipe<true> : k_source_tc_pipe<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntot = (long long)d.ng * nbatch * ((d.nyz + kTN - 1) / kTN);
    long long blocks = lc.num_sms;  // one CTA per SM (shared memory; TMEM up to all 512 columns)
    if (blocks > ntot) blocks = ntot;
    kern<<<(unsigned)blocks, kPipeThreads, smem, lc.stream>>>(ma, mb, src, d.na, d.nyz, d.ng, d.ng * nbatch, nstages,
                                                              (float)dudv, lc.err);
    ++*lc.launches;
    return cudaGetLastError();
  }
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
