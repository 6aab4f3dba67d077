// transport_rows.cuh -- device code of the streaming lateral transport
// substep T(h) (Section 3.4, Eq. distansport; see k_transport_rows.cu for the
// design), shared by the per-substep kernels of k_transport_rows.cu and the
// persistent batch kernel of k_batch.cu.  Everything sits in an unnamed
// namespace: each translation unit that includes it gets its own copy.
#pragma once

#include "pbs_internal.cuh"

namespace pbs {
namespace {
namespace tr {

// Columns per lane: KV = 4, 6 or 8 (a template parameter; 6 fills a warp with
// rows of 96 or 192 columns; 8 spreads the per-row overheads over more
// columns at the cost of registers).
constexpr int kP = 6;        // rows in flight per lane
constexpr int kR = 8;        // ring slots (a power of two >= kP + 1: slot indices wrap by a mask)

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// x with its sign flipped where s is negative (the FP64 limiter).
__device__ __forceinline__ double flip_by(double x, double s) {
  return __longlong_as_double(__double_as_longlong(x) ^ (__double_as_longlong(s) & (long long)0x8000000000000000ULL));
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(a, fmax(b, c)); }

// KV columns of one row.  Elementwise arithmetic goes through the helpers
// below, which issue the packed FP32x2 instructions for float (two columns
// per instruction) and plain ones for double.
template <typename real, int KV>
struct Vk {
  real v[KV];
};

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }

template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> add4(const Vk<real, KV> &a, const Vk<real, KV> &b) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t = __fadd2_rn(pk(a.v[j], a.v[j + 1]), pk(b.v[j], b.v[j + 1]));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = a.v[j] + b.v[j];
  }
  return r;
}
// a - b
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> sub4(const Vk<real, KV> &a, const Vk<real, KV> &b) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t = __ffma2_rn(pk(b.v[j], b.v[j + 1]), pk(-1.f, -1.f), pk(a.v[j], a.v[j + 1]));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = a.v[j] - b.v[j];
  }
  return r;
}
// s * (B + h * sl) with h = 1/2
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> face4(real s, const Vk<real, KV> &B, const Vk<real, KV> &sl) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t =
          __fmul2_rn(pk(s, s), __ffma2_rn(pk(0.5f, 0.5f), pk(sl.v[j], sl.v[j + 1]), pk(B.v[j], B.v[j + 1])));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = s * fma(real(0.5), sl.v[j], B.v[j]);
  }
  return r;
}
// B + sl / 2: the upwind face value (a flux without its speed)
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> fval4(const Vk<real, KV> &B, const Vk<real, KV> &sl) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t = __ffma2_rn(pk(0.5f, 0.5f), pk(sl.v[j], sl.v[j + 1]), pk(B.v[j], B.v[j + 1]));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = fma(real(0.5), sl.v[j], B.v[j]);
  }
  return r;
}
// a + s b
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> axpy4(real s, const Vk<real, KV> &b, const Vk<real, KV> &a) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t = __ffma2_rn(pk(s, s), pk(b.v[j], b.v[j + 1]), pk(a.v[j], a.v[j + 1]));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = fma(s, b.v[j], a.v[j]);
  }
  return r;
}
// s a
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> scale4(real s, const Vk<real, KV> &a) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
#pragma unroll
    for (int j = 0; j < KV; j += 2) {
      const float2 t = __fmul2_rn(pk(s, s), pk(a.v[j], a.v[j + 1]));
      r.v[j] = t.x;
      r.v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < KV; j++) r.v[j] = s * a.v[j];
  }
  return r;
}
// a + (b - c) + e
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> upd4(const Vk<real, KV> &a, const Vk<real, KV> &b, const Vk<real, KV> &c,
                                             const Vk<real, KV> &e) {
  return add4(add4(a, sub4(b, c)), e);
}

// sign(a) xor sign(b) times min(|a|, |b|) (one min/max instruction).
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
  float r;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Superbee slopes of the lane's columns from their differences d1 (behind)
// and d2 (ahead): the packed part (2x, 2|d2|) and the per-column limiter.
// FP32, four min/max-class instructions per column:
//   u = sign(d1 d2) min(2|d1|, |d2|),  w = sign(d1 d2) min(|d1|, 2|d2|)
//   (both >= 0 exactly when d1, d2 agree in sign), m = max(0, u, w), and the
//   slope sign(d2) m = sign(2 d2) min(m, 2|d2|) since m <= 2|d2|: the same
//   values as the form below (the sign flip and copysign are folded into the
//   sign rule of the min).
// FP64: x = d1 sign(d2), m = max(0, min(2x, |d2|), min(x, 2|d2|)), sign(d2) m.
template <typename real, int KV>
__device__ __forceinline__ Vk<real, KV> slope4(const Vk<real, KV> &d1, const Vk<real, KV> &d2) {
  Vk<real, KV> r;
  if constexpr (sizeof(real) == 4) {
    const Vk<real, KV> x2 = add4(d1, d1), t2 = add4(d2, d2);
#pragma unroll
    for (int j = 0; j < KV; j++) {
      const float u = min_xorsign_abs(x2.v[j], d2.v[j]), w = min_xorsign_abs(d1.v[j], t2.v[j]);
      r.v[j] = min_xorsign_abs(max3(0.f, u, w), t2.v[j]);
    }
  } else {
    Vk<real, KV> x, x2, t2;
#pragma unroll
    for (int j = 0; j < KV; j++) x.v[j] = flip_by(d1.v[j], d2.v[j]);
    x2 = add4(x, x);
    t2 = add4(d2, d2);
#pragma unroll
    for (int j = 0; j < KV; j++) {
      const real m = max3(real(0), fmin(x2.v[j], fabs(d2.v[j])), fmin(x.v[j], fabs(t2.v[j])));
      r.v[j] = copysign(m, d2.v[j]);
    }
  }
  return r;
}

// Bytes per cp.async chunk of a lane's KV columns (16 when every lane's chunk
// starts 16-byte aligned, else 8).
template <typename real, int KV>
__host__ __device__ constexpr int row_chunk() {
  return (KV * sizeof(real)) % 16 == 0 ? 16 : 8;
}

// Row I/O in the march frame.  FZ: columns in memory order; otherwise the
// lane -> column map is mirrored (the row is read and written reversed).
template <typename real, bool VEC, bool FZ, int KV>
struct RowIO {
  // Copy row `row` of a plane into the lane's ring slot `dst`.  Mirrored
  // VEC rows land in physical order and are reversed on read.
  static __device__ __forceinline__ void issue(real *dst, const real *plane_base, int row, int nz, int col0, bool on) {
    const real *rowp = plane_base + (long long)row * nz;
    if (VEC) {
      constexpr int CB = row_chunk<real, KV>(), CE = CB / (int)sizeof(real);
      const int pc = FZ ? col0 : nz - KV - col0;  // physical first column of the lane's chunk
      const unsigned nb = on ? (unsigned)CB : 0u;
#pragma unroll
      for (int k = 0; k < KV / CE; k++) {
        if (CB == 16)
          cp_async16(dst + k * CE, on ? rowp + pc + k * CE : plane_base, nb);
        else
          cp_async8(dst + k * CE, on ? rowp + pc + k * CE : plane_base, nb);
      }
    } else {
#pragma unroll
      for (int k = 0; k < KV; k++) {
        const int q = col0 + k;
        const bool in = on && (q < nz);
        const int pcol = FZ ? q : nz - 1 - q;
        if (sizeof(real) == 8)
          cp_async8(dst + k, in ? rowp + pcol : plane_base, in ? 8u : 0u);
        else
          cp_async4(dst + k, in ? rowp + pcol : plane_base, in ? 4u : 0u);
      }
    }
  }
  static __device__ __forceinline__ void read(const real *src, Vk<real, KV> &x) {
#pragma unroll
    for (int k = 0; k < KV; k++) x.v[k] = (VEC && !FZ) ? src[KV - 1 - k] : src[k];
  }
  // VEC store of a lane's KV columns at dst (physical order)
  static __device__ __forceinline__ void store_vec(real *dst, const Vk<real, KV> &x) {
    real y[KV];
#pragma unroll
    for (int k = 0; k < KV; k++) y[k] = FZ ? x.v[k] : x.v[KV - 1 - k];
    if (sizeof(real) == 4 && KV == 4) {
      *reinterpret_cast<float4 *>(dst) = make_float4((float)y[0], (float)y[1], (float)y[2], (float)y[3]);
    } else if (sizeof(real) == 4) {
#pragma unroll
      for (int k = 0; k < KV; k += 2) *reinterpret_cast<float2 *>(dst + k) = make_float2((float)y[k], (float)y[k + 1]);
    } else {
#pragma unroll
      for (int k = 0; k < KV; k += 2)
        *reinterpret_cast<double2 *>(dst + k) = make_double2((double)y[k], (double)y[k + 1]);
    }
  }
  static __device__ __forceinline__ void store(real *plane_base, int row, int nz, int col0, bool on,
                                               const Vk<real, KV> &x) {
    if (!on) return;
    real *rowp = plane_base + (long long)row * nz;
    if (VEC) {
      store_vec(rowp + (FZ ? col0 : nz - KV - col0), x);
    } else {
#pragma unroll
      for (int k = 0; k < KV; k++) {
        const int q = col0 + k;
        if (q < nz) rowp[FZ ? q : nz - 1 - q] = x.v[k];
      }
    }
  }
};

// z contribution (G_lo - G_hi) h/dz for the lane's KV cells of one row in the
// march frame (positive flow).  gz = |v| h / dz.  zl / zr: 0 for the first /
// last lane of the plane (zero ghosts), else 1.
template <typename real, int KV>
__device__ __forceinline__ void z_delta(const Vk<real, KV> &c, real gz, real zl, real zr, int gw, Vk<real, KV> &out) {
  const real lft = zl * __shfl_up_sync(0xffffffffu, c.v[KV - 1], 1, gw);  // the column left of the lane's first
  const real rgt = zr * __shfl_down_sync(0xffffffffu, c.v[0], 1, gw);     // the column right of the lane's last
  // right faces of the lane's cells
  Vk<real, KV> dl, dr;
  dl.v[0] = c.v[0] - lft;
#pragma unroll
  for (int j = 0; j + 1 < KV; j++) dr.v[j] = dl.v[j + 1] = c.v[j + 1] - c.v[j];
  dr.v[KV - 1] = rgt - c.v[KV - 1];
  const Vk<real, KV> g = face4(gz, c, slope4(dl, dr));
  // left face = the left neighbour's last right face; inflow edge: zero ghosts upstream
  const real glo = zl * __shfl_up_sync(0xffffffffu, g.v[KV - 1], 1, gw);
  Vk<real, KV> gl;
  gl.v[0] = glo;
#pragma unroll
  for (int j = 1; j < KV; j++) gl.v[j] = g.v[j - 1];
  out = sub4(gl, g);
}

// As z_delta with unscaled face values: the difference (left face value -
// right face value) of the lane's KV cells, to be multiplied by |v| h / dz.
template <typename real, int KV>
__device__ __forceinline__ void z_delta_v(const Vk<real, KV> &c, real zl, real zr, int gw, Vk<real, KV> &out) {
  const real lft = zl * __shfl_up_sync(0xffffffffu, c.v[KV - 1], 1, gw);
  const real rgt = zr * __shfl_down_sync(0xffffffffu, c.v[0], 1, gw);
  Vk<real, KV> dl, dr;
  dl.v[0] = c.v[0] - lft;
#pragma unroll
  for (int j = 0; j + 1 < KV; j++) dr.v[j] = dl.v[j + 1] = c.v[j + 1] - c.v[j];
  dr.v[KV - 1] = rgt - c.v[KV - 1];
  const Vk<real, KV> g = fval4(c, slope4(dl, dr));
  const real glo = zl * __shfl_up_sync(0xffffffffu, g.v[KV - 1], 1, gw);
  Vk<real, KV> gl;
  gl.v[0] = glo;
#pragma unroll
  for (int j = 1; j < KV; j++) gl.v[j] = g.v[j - 1];
  out = sub4(gl, g);
}

template <typename real, bool VEC, bool FZ, int KV>
struct PlaneMarch {
  using IO = RowIO<real, VEC, FZ, KV>;
  real *ring;  // this lane's ring base (slot stride 32*KV)
  real *pbase;
  int ny, nz, col0, gw, li;  // col0: the lane's first column in the march frame; li: lane in its group
  bool fwd, on, own;     // on: the lane's columns are loaded; own: they are stored
  real sy, gz, zl, zr;
  int rd, wr;
  // VEC rows: the lane's first physical column of march row m sits at
  // lrow0 + m * lstep (loads; a lane that is off re-reads its own plane base
  // with zero fill: lstep = 0) and srow0 + m * sstep (stores)
  const real *lrow0;
  real *srow0;
  long long lstep, sstep;
  unsigned nbytes;

  __device__ __forceinline__ void setup_rows() {
    if (VEC) {
      const int pc = FZ ? col0 : nz - KV - col0;
      const long long r0 = fwd ? 0 : (long long)(ny - 1) * nz;
      const long long st = fwd ? nz : -(long long)nz;
      srow0 = pbase + r0 + pc;
      sstep = st;
      lrow0 = on ? srow0 : pbase;
      lstep = on ? st : 0;
      nbytes = on ? (unsigned)row_chunk<real, KV>() : 0u;
    }
  }
  __device__ __forceinline__ void issue_row(real *dst, int m) {
    if (VEC) {
      const real *src = lrow0 + m * lstep;
      constexpr int CB = row_chunk<real, KV>(), CE = CB / (int)sizeof(real);
#pragma unroll
      for (int k = 0; k < KV / CE; k++) {
        if (CB == 16)
          cp_async16(dst + k * CE, src + k * CE, nbytes);
        else
          cp_async8(dst + k * CE, src + k * CE, nbytes);
      }
    } else {
      IO::issue(dst, pbase, prow(m), nz, col0, on);
    }
  }
  __device__ __forceinline__ void store_row(int m, const Vk<real, KV> &x) {
    if (VEC) {
      if (!own) return;
      IO::store_vec(srow0 + m * sstep, x);
    } else {
      IO::store(pbase, prow(m), nz, col0, own, x);
    }
  }
  Vk<real, KV> w[4], st[4];  // psi rows i-3..i, psi* rows i-4..i-1 (march order)
  Vk<real, KV> f1, f2;       // carried y face values of stage 1 and stage 2 (fluxes for the CN form)
  Vk<real, KV> e1, e2;       // carried y differences of stage 1 and stage 2

  __device__ __forceinline__ int prow(int m) const { return fwd ? m : ny - 1 - m; }

  __device__ __forceinline__ void prologue() {
    setup_rows();
    wr = 0;
    rd = 0;
#pragma unroll
    for (int j = 0; j < kP; j++) {
      if (j < ny) issue_row(ring + wr * 32 * KV, j);
      cp_async_commit();
      wr++;
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int j = 0; j < KV; j++) w[k].v[j] = st[k].v[j] = real(0);
  }

  // One march iteration i.  LOAD: row i exists (i < ny).  S1: stage 1 for
  // row i-1.  S2: stage 2 for row i-2.  FIRST1/FIRST2: the stage's first row
  // (initialise its carried flux).  IN1: row i-1 < ny.
  template <bool LOAD, bool S1, bool FIRST1, bool IN1, bool S2, bool FIRST2>
  __device__ __forceinline__ void iter(int i) {
    cp_async_wait<kP - 1>();
    Vk<real, KV> x;
    if (LOAD) {
      IO::read(ring + rd * 32 * KV, x);
    } else {
#pragma unroll
      for (int j = 0; j < KV; j++) x.v[j] = real(0);
    }
    rd = (rd + 1) & (kR - 1);
    if (i + kP < ny) issue_row(ring + wr * 32 * KV, i + kP);
    cp_async_commit();
    wr = (wr + 1) & (kR - 1);
#pragma unroll
    for (int k = 0; k < 3; k++) w[k] = w[k + 1];
    w[3] = x;

    // face values are kept without their speeds: psi* = psi + sy (F_lo - F_hi) + gz (G_lo - G_hi)
    if (S1) {  // row m = i-1 needs psi(m-2..m+1) = w[0..3]
      if (FIRST1) {
        const Vk<real, KV> d = sub4(w[2], w[1]);
        f1 = fval4(w[1], slope4(sub4(w[1], w[0]), d));  // face m - 1/2
        e1 = d;
      }
      Vk<real, KV> dz, s;
      z_delta_v(w[2], zl, zr, gw, dz);
      const Vk<real, KV> d = sub4(w[3], w[2]);
      const Vk<real, KV> fh = fval4(w[2], slope4(e1, d));  // face m + 1/2
      e1 = d;
      s = axpy4(gz, dz, axpy4(sy, sub4(f1, fh), w[2]));
      if (!IN1 || !VEC) {
#pragma unroll
        for (int j = 0; j < KV; j++)
          if (!(IN1 && (VEC || col0 + j < nz))) s.v[j] = real(0);
      }
      f1 = fh;
#pragma unroll
      for (int k = 0; k < 3; k++) st[k] = st[k + 1];
      st[3] = s;
    }
    if (S2) {  // row m' = i-2 needs psi*(m'-2..m'+1) = st[0..3] and psi(m') = w[1]
      if (FIRST2) {
        const Vk<real, KV> d = sub4(st[2], st[1]);
        f2 = fval4(st[1], slope4(sub4(st[1], st[0]), d));
        e2 = d;
      }
      Vk<real, KV> dz;
      z_delta_v(st[2], zl, zr, gw, dz);
      const Vk<real, KV> d = sub4(st[3], st[2]);
      const Vk<real, KV> fh = fval4(st[2], slope4(e2, d));
      e2 = d;
      const Vk<real, KV> o = scale4(real(0.5), axpy4(gz, dz, axpy4(sy, sub4(f2, fh), add4(w[1], st[2]))));
      f2 = fh;
      store_row(i - 2, o);
    }
  }

  __device__ __forceinline__ void run() {
    prologue();
    if (ny >= 3) {
      iter<true, false, false, true, false, false>(0);
      iter<true, true, true, true, false, false>(1);
      iter<true, true, false, true, true, true>(2);
#pragma unroll 4
      for (int i = 3; i < ny; i++) iter<true, true, false, true, true, false>(i);
      iter<false, true, false, true, true, false>(ny);
      iter<false, true, false, false, true, false>(ny + 1);
    } else if (ny == 2) {
      iter<true, false, false, true, false, false>(0);
      iter<true, true, true, true, false, false>(1);
      iter<false, true, false, true, true, true>(2);
      iter<false, true, false, false, true, false>(3);
    } else {  // ny == 1
      iter<true, false, false, true, false, false>(0);
      iter<false, true, true, true, false, false>(1);
      iter<false, true, false, false, true, true>(2);
    }
  }
};

template <typename real, bool VEC, bool FZ, int KV>
__device__ __forceinline__ void march_plane(real *ring, real *pbase, int ny, int nz, int col0, int gw, bool fwd,
                                            bool on, bool own, real sy, real gz, real zl, real zr) {
  PlaneMarch<real, VEC, FZ, KV> pm;
  pm.ring = ring;
  pm.pbase = pbase;
  pm.ny = ny;
  pm.nz = nz;
  pm.col0 = col0;
  pm.gw = gw;
  pm.fwd = fwd;
  pm.on = on;
  pm.own = own;
  pm.sy = sy;
  pm.gz = gz;
  pm.zl = zl;
  pm.zr = zr;
  pm.run();
}

// The tasks (plane of the class, segment) of warp gwarp out of nwarps warps:
// each lane group of gw lanes marches one task at a time.  ring: this
// warp's ring (kR slots of 32 KV values).  Every copy has landed on return.
// No Crank-Nicolson march: the explicit trapezoid's kernels pass this.
struct NoCnMarch {
  template <typename real>
  __device__ __forceinline__ void operator()(real *, real *, int, int, int, int, int, bool, bool, real, real, real,
                                             real) const {}
};

template <typename real, bool VEC, bool FZ, int KV, bool CN, typename CnMarch>
__device__ __forceinline__ void transport_tasks(real *__restrict__ psi, long long nplanes, int ny, int nz, int na,
                                                int a0, int na_half, int nu, int nv, real du, real dv, real ky,
                                                real kz, int nseg, int seg_w, int gw, int lane, long long gwarp,
                                                long long nwarps, real *ring_warp, CnMarch march_cn) {
  const int ngroups = 32 / gw;
  const int gi = lane / gw;
  real *ring = ring_warp + (size_t)lane * KV;
  const int li = lane % gw;
  const long long ntasks = nplanes * nseg;

  for (long long base = gwarp * ngroups; base < ntasks; base += nwarps * ngroups) {
    const long long task = base + gi;
    const bool valid = task < ntasks;
    const long long idx = valid ? task / nseg : 0;  // plane of this class
    const int seg = valid ? (int)(task - idx * nseg) : 0;
    const long long stack = idx / na_half;
    const int a = a0 + (int)(idx - stack * na_half);
    const long long plane = stack * na + a;
    // owned columns [s0, s1), loaded columns [s0 - left halo, hi)
    const int s0 = seg * seg_w;
    const int s1 = min(nz, s0 + seg_w);
    const int c_lo = seg > 0 ? s0 - KV : 0;
    const int hi = seg < nseg - 1 ? min(nz, s1 + KV) : nz;
    const int lp = (hi - c_lo + KV - 1) / KV;  // lanes of this segment
    const int col0 = c_lo + li * KV;
    const bool on = valid && li < lp;
    const bool own = on && col0 >= s0 && col0 < s1;
    const real zl = li == 0 ? real(0) : real(1);
    const real zr = li >= lp - 1 ? real(0) : real(1);
    const real uu = (real)((a % nu) - 0.5 * (nu - 1)) * du;
    const real vv = (real)((a / nu) - 0.5 * (nv - 1)) * dv;
    real *pbase = psi + plane * (long long)ny * nz;
    if constexpr (CN)
      march_cn(ring, pbase, ny, nz, col0, gw, li, uu >= real(0), on, fabs(uu) * ky, fabs(vv) * kz, zl, zr);
    else
      march_plane<real, VEC, FZ, KV>(ring, pbase, ny, nz, col0, gw, uu >= real(0), on, own, fabs(uu) * ky,
                                     fabs(vv) * kz, zl, zr);
  }
  cp_async_wait<0>();
}

}  // namespace tr
}  // namespace
}  // namespace pbs
