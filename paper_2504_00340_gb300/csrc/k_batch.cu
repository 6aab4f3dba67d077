// k_batch.cu -- the depth march of a whole batch of pencil beams (spots) in
// one persistent launch.
//
// Each beam is its own context (own grid, energy groups, tables, density and
// workspace).  Its march is a chain of passes over its psi: per depth step s
// the Strang sequence of Section 3.3 as four passes,
//   E(h/2) [closing step s-1, fused with opening step s]   T(h/2)   A(h)   T(h/2),
// and after its last step the closing E(h/2).  Each pass splits into tiles:
// the blocks of the per-substep kernels (the same device code, energy_f2.cuh,
// transport_rows.cuh, angular_f2.cuh), so a tile computes exactly what the
// corresponding block of the ordinary launch computes.
//
// The queue is a host-built list of (beam, pass) tasks, round-robin over the
// beams (pass 0 of every beam, then pass 1 of every beam still marching, ...).
// The CTAs of one persistent launch hand out the tiles of the current task
// through its counter and advance the task index when it runs dry, so tiles
// leave the queue in task order.  A tile of pass p of beam b waits until b's
// completion counter has reached the number of b's tiles in passes before p;
// every tile it waits for left the queue earlier, to a CTA that is running
// and whose own wait is on still earlier tiles, so the waits always end.
// Each wait is bounded (SM clocks): a wait that gives up sets the batch abort
// word and every beam's device status word, and every CTA stops at its next
// tile boundary, with nothing in flight.
#include "pbs_internal.cuh"
#include "angular_f2.cuh"
#include "energy_f2.cuh"
#include "transport_rows.cuh"

#include <algorithm>

namespace pbs {

namespace {

using namespace batch_pass;

// CTA shapes (pbs_batch_options.shape), both 16 warps' worth of work per SM:
//   0  256 threads, two CTAs per SM at 128 registers: an energy block of
//      32 x 8 threads (16 angles x 64 lateral points), eight transport warps
//      (4 columns per lane), two angular sub-blocks of 16 x 8;
//   1  128 threads, three CTAs per SM at up to 170 registers: an energy block
//      of 32 x 4 (8 angles), four transport warps (4 or 6 columns: the
//      6-column march needs ~144 registers), one angular sub-block.
// The angular tile needs few registers but many loads in flight, so each
// sub-block works on four independent slab stacks at a time.
template <int SHAPE>
struct BShape {
  static constexpr int kThreads = SHAPE == 0 ? 256 : 128;
  static constexpr int kMinBlocks = SHAPE == 0 ? 2 : 3;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kEnergyY = kThreads / 32;
};
// Angular sub-blocks of 16 x NT threads per CTA (16 x 16 angles need a whole
// 256-thread CTA), and slab stacks worked at a time per sub-block.
template <int SHAPE, int NT>
__host__ __device__ constexpr int ang_subs() { return BShape<SHAPE>::kThreads / (16 * NT); }
template <int NT>
__host__ __device__ constexpr int ang_r() { return NT <= 8 ? 4 : 1; }
constexpr int kBAngRep = 32;    // angular slab stacks per tile (and per chunk of a pipelined pass)

// Ask the L2 for the rows of R slab stacks kgc0 + r (r < R, those < nkgc) at
// lateral block bx: one hint per 128-byte line (16 threads share a line).
template <int NU, int NV, int R>
__device__ __forceinline__ void prefetch_stacks(const float *psi, int nyz, long long kgc0, long long nkgc, int bx,
                                                int x, int t) {
  if (x != 0 || t >= NV) return;
  const int yz = bx * ang::kF2X * 2;
  if (yz >= nyz) return;
#pragma unroll
  for (int r = 0; r < R; r++) {
    if (kgc0 + r >= nkgc) break;
    const float *base = psi + (kgc0 + r) * (long long)(NU * NV) * nyz + yz;
#pragma unroll
    for (int i = 0; i < NU; i++)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (long long)(t * NU + i) * nyz));
  }
}


__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Give up the whole batch: the abort word, and every beam's status word.
__device__ void batch_abort(const BatchBeam *beams, int nbeams, int *abort_word, int where) {
  if (atomicCAS(abort_word, 0, where) == 0) {
    for (int b = 0; b < nbeams; b++) {
      if (beams[b].err) {
        atomicAdd(beams[b].err, 1);
        atomicExch(beams[b].err + 1, kErrTimeoutBatch);
      }
    }
  }
}

// One sweep of 16 x 16 angular stacks as a separate function: inlined
// into the persistent loop, their sine-table operands are hoisted out of the
// loop into registers and the tile spills (~1 KB per thread at 128
// registers); called, it needs no spill.  (Angle grids of at most 8 x 8 stay
// inlined: there the call costs more than it saves.)
template <int NU, int NV, int R>
__device__ __noinline__ void angular_sweep(float *psi, const float *rho_yz, const float *ts, int nyz, int ng, float hq,
                                           long long kgc0, long long nkgc, int bx, int x, int t, unsigned char *sm,
                                           const ang::AngTables<float> &tb) {
  ang::angular_f2_tiles<NU, NV, false, R, true>(psi, rho_yz, ts, nyz, ng, hq, kgc0, 1, nkgc, bx, x, t, sm, tb);
}

template <int NU, int NV, int SHAPE>
__device__ __forceinline__ void run_tile(const BatchBeam &bm, const BatchTask &tk, long long tile, unsigned char *smem,
                                         const ang::AngTables<float> &tb) {
  const int kind = tk.kind, step = tk.step;
  using S = BShape<SHAPE>;
  const Dims &d = bm.d;
  const int tid = threadIdx.x;
  const size_t nyz = (size_t)d.nyz;
  if (kind == kPassEOpen || kind == kPassEPair || kind == kPassEClose) {
    const int bx = (int)(tile % bm.e_bx), by = (int)(tile / bm.e_bx);
    const BeamStrides bs{0, 0, 0, 0};
    // E(h/2) with the density of slab sa: opening step 0, closing the last
    // step, or closing step - 1 fused with opening step (its slab), with the
    // fluence after the closing half
    const int sa = kind == kPassEOpen ? 0 : step - 1;
    if (kind == kPassEPair) {
      en::energy_f2_tile<float, false, false, true, S::kEnergyY>(
          bx, by, 0, tid & 31, tid >> 5, smem, d, bm.psi, nullptr, nullptr, nullptr, nullptr, bm.rho + sa * nyz,
          bm.rho + (size_t)step * nyz, bm.coef, bm.dose + sa * nyz, bm.dose + (size_t)step * nyz,
          bm.flu + (size_t)step * nyz, bm.c, bm.c, bm.dose_scale, bm.flu_scale, bs);
    } else {
      double *flu = kind == kPassEClose ? bm.flu + (size_t)bm.n_steps * nyz : nullptr;
      en::energy_f2_tile<float, false, false, false, S::kEnergyY>(
          bx, by, 0, tid & 31, tid >> 5, smem, d, bm.psi, nullptr, nullptr, nullptr, nullptr, bm.rho + sa * nyz,
          nullptr, bm.coef, bm.dose + sa * nyz, nullptr, flu, bm.c, bm.c, bm.dose_scale, bm.flu_scale, bs);
    }
  } else if (kind == kPassT) {
    // one slab stack (component, g, c) of one mirror class per tile: the
    // task's stacks of the class v < 0, then of the class v >= 0
    const long long nst = tk.nstacks;
    const int fz = tile >= nst ? 1 : 0;
    const long long stack = tk.first + (fz ? tile - nst : tile);
    const int a_split = (d.nv / 2) * d.nu;
    const int a0 = fz ? a_split : 0, na_half = fz ? d.na - a_split : a_split;
    float *psi = bm.psi + stack * (long long)d.na * d.nyz;
    const int lane = tid & 31, warp = tid >> 5;
#define PBS_BT(KV, FZ)                                                                                            \
  tr::transport_tasks<float, true, FZ, KV, false>(psi, na_half, d.ny, d.nz, d.na, a0, na_half, d.nu, d.nv, bm.du, \
                                                  bm.dv, bm.ky, bm.kz, bm.tr_nseg, bm.tr_segw, bm.tr_gw, lane,   \
                                                  warp, S::kWarps,                                                \
                                                  reinterpret_cast<float *>(smem) + (size_t)warp * tr::kR * 32 * KV, \
                                                  tr::NoCnMarch{})
    if (SHAPE == 1 && bm.tr_kv == 6) {
      if (fz) PBS_BT(6, true); else PBS_BT(6, false);
    } else {
      if (fz) PBS_BT(4, true); else PBS_BT(4, false);
    }
#undef PBS_BT
  } else {  // kPassA: kBAngRep consecutive slab stacks of the task at one lateral block
    constexpr int NT = NU > NV ? NU : NV;
    constexpr int kSub = ang_subs<SHAPE, NT>(), kR = ang_r<NT>();
    const int bx = (int)(tile % bm.a_bx);
    const long long k0 = tk.first + (tile / bm.a_bx) * kBAngRep;
    const long long kend = tk.first + tk.nstacks;  // the task's stacks end here
    constexpr int kPer = kSub * kR;  // stacks per sweep of the CTA
    const int sub = tid / (16 * NT);
    const int x = tid & 15, t = (tid >> 4) % NT;
    unsigned char *sm = smem + (size_t)sub * kR * sizeof(float2) * NU * NV * ang::kF2X;
#pragma unroll 1
    for (int it = 0; it < kBAngRep / kPer && k0 + kPer * it < kend; it++) {
      // the next sweep's rows travel to the L2 while this sweep computes
      if (it + 1 < kBAngRep / kPer)
        prefetch_stacks<NU, NV, kR>(bm.psi, d.nyz, k0 + kPer * (it + 1) + kR * sub, kend, bx, x, t);
      if constexpr (NT == 16)
        angular_sweep<NU, NV, kR>(bm.psi, bm.rho + (size_t)step * nyz, bm.ts, d.nyz, d.ng, bm.hq,
                                  k0 + kPer * it + kR * sub, kend, bx, x, t, sm, tb);
      else
        ang::angular_f2_tiles<NU, NV, false, kR, true>(bm.psi, bm.rho + (size_t)step * nyz, bm.ts, d.nyz, d.ng,
                                                       bm.hq, k0 + kPer * it + kR * sub, 1, kend, bx, x, t, sm, tb);
      __syncthreads();  // the next stacks reuse the shared tiles
    }
  }
}

template <int NU, int NV, int SHAPE>
__global__ void __launch_bounds__(BShape<SHAPE>::kThreads, BShape<SHAPE>::kMinBlocks)
    k_batch(const BatchBeam *__restrict__ beams, int nbeams, const BatchTask *__restrict__ tasks, int ntasks,
            BatchQueue *q, unsigned long long *done_ctr, unsigned long long *next_ctr, long long wait_cycles,
            unsigned long long *prof, const __grid_constant__ ang::AngTables<float> tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task, s_go;
  __shared__ long long s_tile;
  const int tid = threadIdx.x;
  long long t_claim = 0, t_start = 0;
  for (;;) {
    if (tid == 0) {
      if (prof) t_claim = clock64();
      int go = 0, t = 0;
      long long tile = 0;
      for (;;) {
        if (ld_acquire_i(&q->abort) != 0) break;
        t = (int)ld_acquire(&q->cur);
        if (t >= ntasks) break;
        tile = (long long)atomicAdd(&next_ctr[t], 1ULL);
        if (tile < tasks[t].ntiles) {
          go = 1;
          break;
        }
        atomicCAS(&q->cur, (unsigned long long)t, (unsigned long long)t + 1);  // this task is handed out
      }
      if (go && tasks[t].wait_ctr >= 0) {
        // the tiles this task depends on (all of them earlier in the queue) have completed
        const BatchTask tk = tasks[t];
        const unsigned long long need = (unsigned long long)tk.wait_need;
        unsigned long long *done = &done_ctr[tk.wait_ctr];
        if (ld_acquire(done) < need) {
          const long long t0 = clock64();
          while (ld_acquire(done) < need) {
            if (ld_acquire_i(&q->abort) != 0) {
              go = 0;
              break;
            }
            if (clock64() - t0 > wait_cycles) {
              batch_abort(beams, nbeams, &q->abort, 1 + tk.beam);
              go = 0;
              break;
            }
            __nanosleep(200);
          }
        }
      }
      s_task = t;
      s_tile = tile;
      s_go = go;
      if (prof) {
        t_start = clock64();
        atomicAdd(&prof[3], (unsigned long long)(t_start - t_claim));
      }
    }
    __syncthreads();
    if (!s_go) break;
    const BatchTask tk = tasks[s_task];
    const BatchBeam &bm = beams[tk.beam];
    run_tile<NU, NV, SHAPE>(bm, tk, s_tile, smem, tb);
    __syncthreads();  // every thread's writes of this tile are done
    if (tid == 0) {
      __threadfence();
      atomicAdd(&done_ctr[tk.sig_ctr], 1ULL);
      if (prof) {
        const int k = tk.kind == kPassT ? 1 : (tk.kind == kPassA ? 2 : 0);
        atomicAdd(&prof[k], (unsigned long long)(clock64() - t_start));
        atomicAdd(&prof[4 + k], 1ULL);
      }
    }
  }
}

template <int NU, int NV, int SHAPE>
cudaError_t go_batch(const LaunchCtx &lc, const BatchBeam *beams, int nbeams, const BatchTask *tasks, int ntasks,
                     BatchQueue *q, unsigned long long *done, unsigned long long *next, long long wait_cycles,
                     size_t smem, double du, double dv, unsigned long long *prof, int *ctas) {
  auto kern = k_batch<NU, NV, SHAPE>;
  constexpr int kThreads = BShape<SHAPE>::kThreads;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  ang::AngTables<float> tb;
  ang::fill_tables(tb, NU, NV, du, dv);
  // A CTA only ever waits for tiles that left the queue before its own, that
  // is, for tiles held by CTAs already running: the launch needs no
  // co-residency guarantee (and so stays capturable in a graph).
  *ctas = per_sm * lc.num_sms;
  kern<<<(unsigned)(per_sm * lc.num_sms), kThreads, smem, lc.stream>>>(beams, nbeams, tasks, ntasks, q, done, next,
                                                                        wait_cycles, prof, tb);
  ++*lc.launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t batch_init_tables() { return ang::upload_dst_f2(); }

// Transport columns per lane of a beam: want = 4 or 6 (6 where rows split
// evenly into 6-column lanes, else 4), or 0 for the per-substep kernel's
// default rule: 6 where that fills the warps better than 4.
static int batch_kv(int nz, int want, int &nseg, int &seg_w, int &gw) {
  auto use = [&](int kv, int &ns, int &sw, int &g) {
    int lanes;
    if (nz <= 32 * kv) {
      ns = 1;
      sw = nz;
      lanes = (nz + kv - 1) / kv;
    } else {  // rows cut into segments as in the per-substep kernel
      const int wmax = (32 - 2) * kv;
      ns = (nz + wmax - 1) / wmax;
      sw = ((nz + ns - 1) / ns + kv - 1) / kv * kv;
      lanes = sw / kv + 2;
    }
    g = 1;
    while (g < lanes) g <<= 1;
    return (double)nz / ((double)ns * g * kv);
  };
  int n4, s4, g4, n6 = 1, s6 = 0, g6 = 1;
  const double u4 = use(4, n4, s4, g4);
  const double u6 = (want != 4 && nz % 6 == 0) ? use(6, n6, s6, g6) : 0.0;
  if (want == 6 ? u6 > 0.0 : (want == 0 && u6 > u4 + 0.05)) {
    nseg = n6; seg_w = s6; gw = g6;
    return 6;
  }
  nseg = n4; seg_w = s4; gw = g4;
  return 4;
}

BatchShape batch_shape(const Dims &d, int shape, int cols) {
  BatchShape s{};
  const int threads = shape == 0 ? BShape<0>::kThreads : BShape<1>::kThreads;
  const int ey = threads / 32, warps = threads / 32;
  s.e_bx = (d.nyz / 2 + en::kX - 1) / en::kX;
  s.e_by = (d.na + ey * en::kA - 1) / (ey * en::kA);
  s.e_tiles = (long long)s.e_bx * s.e_by;
  s.tr_stacks = (long long)d.ncomp * d.ng * 2;
  s.t_tiles = 2 * s.tr_stacks;
  // 6 columns only on the shape with the registers for it, and where rows
  // split evenly into 6-column lanes
  const int want = shape == 1 ? cols : 4;
  s.tr_kv = batch_kv(d.nz, want, s.tr_nseg, s.tr_segw, s.tr_gw);
  s.a_bx = (d.nyz / 2 + ang::kF2X - 1) / ang::kF2X;
  s.a_tiles = (long long)s.a_bx * (((long long)d.ncomp * d.ng * 2 + kBAngRep - 1) / kBAngRep);
  const int nt = std::max(d.nu, d.nv);
  const int subs = std::max(1, threads / (16 * nt)), r = nt <= 8 ? 4 : 1;
  s.smem = std::max(sizeof(en::GroupPair) * (size_t)d.ng,
                    std::max((size_t)warps * tr::kR * 32 * s.tr_kv * sizeof(float),
                             (size_t)subs * r * sizeof(float2) * (size_t)d.nu * d.nv * ang::kF2X));
  return s;
}

bool batch_supported(int nu, int nv) { return nu == nv && (nu <= 8 || nu == 16) && angular_supported(nu, nv); }

cudaError_t launch_batch(const LaunchCtx &lc, int shape, int nu, int nv, const BatchBeam *beams, int nbeams,
                         const BatchTask *tasks, int ntasks, BatchQueue *q, unsigned long long *done,
                         unsigned long long *next, long long wait_cycles, size_t smem, double du, double dv,
                         unsigned long long *prof, int *ctas) {
#define PBS_B(A, B)                                                                                           \
  if (nu == A && nv == B)                                                                                     \
    return shape == 0 ? go_batch<A, B, 0>(lc, beams, nbeams, tasks, ntasks, q, done, next, wait_cycles, smem, \
                                          du, dv, prof, ctas)                                                 \
                      : go_batch<A, B, 1>(lc, beams, nbeams, tasks, ntasks, q, done, next, wait_cycles, smem, \
                                          du, dv, prof, ctas);
  PBS_B(2, 2) PBS_B(4, 4) PBS_B(6, 6) PBS_B(8, 8)
#undef PBS_B
  // 16 x 16 angles: a whole 256-thread CTA per angular block (shape 0 only)
  if (nu == 16 && nv == 16 && shape == 0)
    return go_batch<16, 16, 0>(lc, beams, nbeams, tasks, ntasks, q, done, next, wait_cycles, smem, du, dv, prof, ctas);
  return cudaErrorNotSupported;
}

}  // namespace pbs
