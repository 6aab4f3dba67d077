// pbs_api.cu -- C ABI of the library (include/pbs.h): context, caller-bound
// workspace, FP64 host tables, beam projection and the depth-march driver.
//
// Per depth step s (Section 3.3, Strang splitting with Crank-Nicolson in each
// subsystem) every component k = 0..K goes through
//   E(h/2)  T(h/2)  A(h)  T(h/2)  E(h/2)
// with the density of slab s.  In each E substep the components run in
// order; component k (k >= 1) takes the catastrophic source of component
// k-1 (Section 3.1, Eq. pri-se; Remark 1) evaluated at the start and end of
// the same substep (trapezoid), which the energy kernel of k-1 emits fused as
// R and the contraction kernel turns into src = du dv P^2_g R.
//
// A context may hold n_beams independent beams (a batch of spots on one
// grid).  Beam b owns components b*(K+1) .. b*(K+1)+K, its own R/src slots,
// dose and fluence; every kernel launch covers all beams still inside their
// depth range.  Beams are ordered by non-increasing depth (pbs_set_beam_steps)
// so the active ones at any depth form a prefix and the launches shrink as
// beams stop.
#include "pbs_internal.cuh"
#include "pbs.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pbs;
using namespace pbs::batch_pass;

struct pbs_ctx {
  int dev = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  int precision = PBS_FP32;
  int ny, nz, ng, nu, nv, na, nx, K;
  int B = 1;                       // beams held by the context
  std::vector<int> beam_steps;     // depth steps of each beam (non-increasing)
  double dy, dz, dx, u_max, v_max, du, dv;
  std::vector<double> e_faces, e_c, de;
  Dims d;
  // FP64 host tables
  std::vector<double> s_face, ts, sig, p1, p2, q1, decay, u, v;
  // energy straggling: coefficient at the faces, and the stopping power
  // before the drift T'/2 is folded into s_face
  std::vector<double> t_face, s_base;
  bool strag = false;
  double rho_max = 0.0;      // densest voxel of the material (explicit straggling bound)
  double strag_bound = 0.0;  // Gershgorin row bound of the straggling blocks
  bool have_tables = false, have_material = false, have_beam = false;
  // lateral part of a beam decomposed along y (pbs_set_lateral_part): rows
  // 0..ny-1 of this context are rows part_y0..part_y0+ny-1 of a grid of
  // part_nyg rows; the first halo_lo and the last halo_hi rows are copies of
  // the neighbouring parts' rows, refreshed before every transport substep
  bool part = false;
  int part_y0 = 0, part_nyg = 0, halo_lo = 0, halo_hi = 0;
  int stage = 0;                    // next stage of the staged step (pbs_step_stage)
  cudaEvent_t xev = nullptr;        // orders halo copies between parts on different streams
  // persistent batch led by this context (pbs_run_batch): the key of the
  // descriptors last uploaded, and the recorded graph of the batch
  unsigned long long batch_key = 0;
  cudaGraphExec_t batch_graph = nullptr;
  long long batch_graph_kernels = 0;
  // tile-kind clocks of the last profiled batch (device counters, not yet folded)
  const unsigned long long *batch_prof = nullptr;
  int batch_ctas = 0;
  unsigned long long material_hash = 0;  // FNV-1a of the density last set (checkpoint consistency)
  int n_slabs = 0;
  int steps_done = 0;
  bool pending = false;  // closing E(h/2) of the last step not applied yet
  // workspace
  unsigned char *ws = nullptr;
  size_t ws_bytes = 0;
  size_t off_psi, off_r, off_s, off_rho, off_dose, off_flu, off_coef, off_strag, off_omega, off_dinv, off_ts, off_p2,
      off_init, off_err, total;
  size_t rsize, ssize;  // element sizes of real and of the source storage
  long long launches = 0;
  // launch shapes (pbs_autotune / pbs_set_tuning)
  pbs_tuning tune{8, 1, 0, 0, 5, 1};
  pbs_options opts{0, 0, 0};
  // whole-march CUDA graph (pbs_run with use_graph)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_depth = -1;
  long long graph_kernels = 0;
  bool capturing = false;
  std::string err;
  // per-kernel timing (pbs_set_profiling): event pairs recorded on the stream
  struct Rec { int kind; cudaEvent_t a, b; };
  bool profiling = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  long long prof_count[PBS_KERNEL_KINDS] = {};
  double prof_ms[PBS_KERNEL_KINDS] = {};
  ~pbs_ctx() {
    for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (xev) cudaEventDestroy(xev);
    if (batch_graph) cudaGraphExecDestroy(batch_graph);
  }
};

namespace {

pbs_status fail(pbs_ctx *c, pbs_status st, const std::string &msg) {
  if (c) c->err = msg;
  return st;
}

pbs_status cuda_fail(pbs_ctx *c, cudaError_t e, const char *where) {
  return fail(c, PBS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PBS_CUDA(c, call)                                \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Rows a lateral part needs from each neighbour before a transport substep:
// the two stages of the explicit trapezoid each reach two cells upstream
// (upwind-biased limited reconstruction), so a cell's update depends on the
// four rows on either side of it (either side: the speed's sign varies).
constexpr int kHaloRows = 4;

size_t init_stride(const pbs_ctx *c) { return (size_t)(2 * c->ng + c->na + c->ny + c->nz); }

void layout(pbs_ctx *c) {
  const size_t S = c->rsize, SS = c->ssize, B = (size_t)c->B;
  const size_t nyz = (size_t)c->ny * c->nz;
  size_t o = 0;
  c->off_psi = o; o = align256(o + (size_t)c->d.ncomp * c->d.comp_elems * S);
  const size_t nsrc = (c->K > 0) ? (size_t)c->ng * c->na * nyz : 0;
  // R and src: [half][beam][g][a][yz]; half 0/1 = first/second substep of a fused pair
  c->off_r = o; o = align256(o + 2 * B * nsrc * SS);
  c->off_s = o; o = align256(o + 2 * B * nsrc * SS);
  c->off_rho = o; o = align256(o + (size_t)c->nx * nyz * S);
  c->off_dose = o; o = align256(o + B * c->nx * nyz * 8);       // [beam][slab][yz]
  c->off_flu = o; o = align256(o + B * (c->nx + 1) * nyz * 8);  // [beam][plane][yz]
  c->off_coef = o; o = align256(o + (size_t)c->ng * 10 * S);
  c->off_strag = o; o = align256(o + (size_t)c->ng * 12 * S);
  c->off_omega = o; o = align256(o + (size_t)c->ng * 2 * S);          // column weights of the CN straggling dose
  c->off_dinv = o; o = align256(o + (size_t)c->ng * 4 * nyz * S);     // eliminated blocks, [g][4][yz]
  c->off_ts = o; o = align256(o + (size_t)c->ng * S);
  c->off_p2 = o; o = align256(o + ((c->K > 0) ? (size_t)c->ng * c->na * c->na * SS : 0));
  c->off_init = o; o = align256(o + B * init_stride(c) * 8);  // beam projection factors per beam
  c->off_err = o; o = align256(o + 64);
  c->total = o;
}

template <typename T>
T *at(pbs_ctx *c, size_t off) { return reinterpret_cast<T *>(c->ws + off); }

LaunchCtx lctx(pbs_ctx *c) {
  LaunchCtx lc{c->stream, c->num_sms, &c->launches, at<int>(c, c->off_err)};
  lc.energy_angles = c->tune.energy_angles;
  lc.energy_form = c->tune.energy_form;
  lc.transport_ctas = c->tune.transport_ctas;
  lc.transport_cols = c->tune.transport_cols;
  lc.angular_form = c->tune.angular_form;
  lc.source_form = c->tune.source_form;
  lc.angular_exact = c->opts.angular_integrator;
  lc.transport_cn = c->opts.transport_integrator;
  return lc;
}

// Dims of the first nb beams (the active prefix).
Dims dims_for(const pbs_ctx *c, int nb) {
  Dims d = c->d;
  d.nbeam = nb;
  d.ncomp = nb * (c->K + 1);
  return d;
}

// Depth steps of beam b, capped by the material's extent.
int beam_depth(const pbs_ctx *c, int b) { return std::min(c->beam_steps[b], c->n_slabs); }

// Beams still marching at depth step s: a prefix, since depths are non-increasing.
int active_at(const pbs_ctx *c, int s) {
  int n = 0;
  while (n < c->B && beam_depth(c, n) > s) n++;
  return n;
}

int max_depth(const pbs_ctx *c) { return c->B > 0 ? beam_depth(c, 0) : 0; }

void drop_graph(pbs_ctx *c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_depth = -1;
}

cudaEvent_t take_event(pbs_ctx *c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch with an event pair when profiling is on.
struct ProfScope {
  pbs_ctx *c;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(pbs_ctx *c_, int k) : c(c_), kind(k) {
    if (c->profiling && !c->capturing) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (c->profiling && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->recs.push_back({kind, a, b});
    }
  }
};

pbs_status fold_profile(pbs_ctx *c) {
  if (c->batch_prof) {  // a profiled persistent batch: its tile-kind clocks per CTA
    unsigned long long v[8] = {};
    PBS_CUDA(c, cudaMemcpyAsync(v, c->batch_prof, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    PBS_CUDA(c, cudaStreamSynchronize(c->stream));
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->dev) != cudaSuccess || khz <= 0) khz = 2000000;
    const int kinds[4] = {PBS_KERNEL_ENERGY, PBS_KERNEL_TRANSPORT, PBS_KERNEL_ANGULAR, PBS_KERNEL_QUEUE};
    for (int k = 0; k < 4; k++) {
      c->prof_ms[kinds[k]] += (double)v[k] / ((double)c->batch_ctas * khz);
      if (k < 3) c->prof_count[kinds[k]] += (long long)v[4 + k];
    }
    c->batch_prof = nullptr;
  }
  if (c->recs.empty()) return PBS_OK;
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  for (auto &r : c->recs) {
    float ms = 0.f;
    PBS_CUDA(c, cudaEventElapsedTime(&ms, r.a, r.b));
    c->prof_count[r.kind]++;
    c->prof_ms[r.kind] += ms;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  return PBS_OK;
}

// ---------------------------------------------------------------- host tables

// Mass stopping power of the Bragg-Kleeman range law R(E) = alpha E^p:
// S(E) = 1 / R'(E).
double stopping_bk(const pbs_physics &ph, double e) {
  return ph.s_scale / (ph.bk_alpha * ph.bk_p * std::pow(e, ph.bk_p - 1.0));
}

// Primitive of the Highland scattering power (Es / pv)^2 / X0 in E, with
// pv = E (E + 2M) / (E + M):  (Es^2/X0) [ ln(E/(E+2M)) / (4M) - (E+M) / (2E(E+2M)) ].
double highland_primitive(const pbs_physics &ph, double e) {
  const double m = ph.mp;
  return ph.es * ph.es / ph.x0 * (std::log(e / (e + 2.0 * m)) / (4.0 * m) - (e + m) / (2.0 * e * (e + 2.0 * m)));
}

// The paper's own physics for water (Appendix A.1, A.3): Bethe-Bloch per
// element (density correction 0) with the piecewise I-value rule, Bragg
// additivity over the mass fractions, and the screened-Rutherford
// momentum-transfer cross section per atom.
struct Element {
  double z, a, w;  // atomic number, molar mass (g/mol), mass fraction in water
};
constexpr Element kWater[2] = {{1.0, 1.00794, 0.111894}, {8.0, 15.9994, 0.888106}};
constexpr double kMeC2 = 0.51099895;      // MeV
constexpr double kBetheK = 0.307075;      // MeV cm^2 / mol
constexpr double kCoulomb = 1.439964e-13;  // e^2 / (4 pi eps0), MeV cm
constexpr double kFineStructure = 1.0 / 137.035999;
constexpr double kAvogadro = 6.02214076e23;
constexpr double kMeVPerAmu = 931.494;

double excitation_mev(double z) {
  if (z < 1.5) return 19.0e-6;
  return (z <= 13.0 ? 11.2 + 11.7 * z : 52.8 + 8.71 * z) * 1e-6;
}

double stopping_bethe_water(const pbs_physics &ph, double e) {
  const double gam = 1.0 + e / ph.mp, beta2 = 1.0 - 1.0 / (gam * gam);
  double s = 0.0;
  for (const Element &el : kWater)
    s += el.w * kBetheK * el.z / el.a / beta2 *
         (std::log(2.0 * kMeC2 * beta2 * gam * gam / excitation_mev(el.z)) - beta2);
  return ph.s_scale * s;
}

// rho sigma_tr per unit density (cm^2/g): sum over the atoms of one gram.
double scattering_rutherford_water(const pbs_physics &ph, double e) {
  const double gam = 1.0 + e / ph.mp, beta2 = 1.0 - 1.0 / (gam * gam);
  const double p = std::sqrt(e * (e + 2.0 * ph.mp));
  double s = 0.0;
  for (const Element &el : kWater) {
    const double m_target = el.a * kMeVPerAmu;
    const double m_red = ph.mp * m_target / (ph.mp + m_target);
    const double r = el.z * kCoulomb / (m_red * beta2);
    const double theta_min = std::cbrt(el.z) * kFineStructure * kMeC2 / p;
    const double eta = theta_min * theta_min;
    const double sigma = 2.0 * 3.14159265358979323846 * r * r * (std::log((eta + 1.0) / eta) - 1.0 / (eta + 1.0));
    s += kAvogadro * el.w / el.a * sigma;
  }
  return s;
}

double gamma_density(double th, double al, double be) {
  if (!(th > 0.0)) return al == 1.0 ? be : 0.0;
  return std::exp(al * std::log(be) + (al - 1.0) * std::log(th) - be * th - std::lgamma(al));
}

// Straggling coefficient of water per gram (Appendix A.2): Bohr's
// 4 pi e^4 per electron with Williams' binding factor
// 1 + 4 I / (3 m_e v^2) ln(2 m_e v^2 / I), m_e v^2 = m_e c^2 beta^2, for the
// electrons of each element (N_A Z / A per gram, its own I-value).
double straggling_williams_water(const pbs_physics &ph, double e) {
  const double gam = 1.0 + e / ph.mp, mv2 = kMeC2 * (1.0 - 1.0 / (gam * gam));
  const double bohr = 4.0 * 3.14159265358979323846 * kCoulomb * kCoulomb * kAvogadro;  // MeV^2 cm^2 / mol
  double s = 0.0;
  for (const Element &el : kWater) {
    const double i = excitation_mev(el.z);
    s += el.w * el.z / el.a * (1.0 + 4.0 * i / (3.0 * mv2) * std::log(2.0 * mv2 / i));
  }
  return bohr * s;
}

// The drift half of the straggling term, (rho/2) d/dE(T' psi), is the
// stopping-power operator with S replaced by T'/2: fold it into the face
// stopping powers.  T is linear in each group; T' at an inner face is the
// mean of the slopes of its two groups, at an outer face its one group's.
void fold_straggling(pbs_ctx *c) {
  const int G = c->ng;
  c->s_face.assign(G + 1, 0.0);
  c->strag = false;
  for (int f = 0; f <= G; f++) {
    const double lo = f > 0 ? (c->t_face[f] - c->t_face[f - 1]) / c->de[f - 1] : 0.0;
    const double hi = f < G ? (c->t_face[f + 1] - c->t_face[f]) / c->de[f] : 0.0;
    const double slope = (f == 0) ? hi : (f == G ? lo : 0.5 * (lo + hi));
    c->s_face[f] = c->s_base[f] + 0.5 * slope;
    c->strag = c->strag || c->t_face[f] != 0.0;
  }
}

// Blocks of the interior-penalty part (rho/2) d/dE(T dpsi/dE) for group g,
// per unit density and times 2 (StragCoef).  Face f between groups a (below)
// and b = a + 1 (above) adds, with the traces psi^-_f = p1_a + p2_a,
// psi^+_f = p1_b - p2_b, the jump J = psi^- - psi^+, the flux average
// F = T_f (p2_a / dE_a + p2_b / dE_b) and the penalty s = 2 T_f / h_f
// (alpha = (1+1)^2/2, h_f the mean width of a and b):
//   to row 1 of a:  (F - s J) / dE_a          to row 1 of b:  -(F - s J) / dE_b
//   to row 2 of a:  3 (F + (T_f / dE_a - s) J) / dE_a
//   to row 2 of b:  3 (F + (T_f / dE_b - s) J) / dE_b
// and each group adds -12 Tbar_g p2_g / dE_g^2 to its row 2 (the volume
// term, Tbar_g the mean of its face values).  Outer faces carry nothing.
void strag_blocks(const pbs_ctx *c, int g, double out[12]) {
  const int G = c->ng;
  double *lo = out, *dd = out + 4, *up = out + 8;
  for (int i = 0; i < 12; i++) out[i] = 0.0;
  const double de = c->de[g];
  dd[3] -= 12.0 * 0.5 * (c->t_face[g] + c->t_face[g + 1]) / (de * de);
  // side 0: the face above g (g is side a, the neighbour b = g + 1 fills up);
  // side 1: the face below g (g is side b, the neighbour a = g - 1 fills lo)
  for (int side = 0; side < 2; side++) {
    const int f = side == 0 ? g + 1 : g;
    if (f <= 0 || f >= G) continue;
    const int ga = f - 1, gb = f;
    const double t = c->t_face[f], da = c->de[ga], db = c->de[gb];
    const double pen = 2.0 * t / (0.5 * (da + db));
    // F and J as linear forms on (p1_a, p2_a, p1_b, p2_b)
    const double F[4] = {0.0, t / da, 0.0, t / db};
    const double J[4] = {1.0, 1.0, -1.0, 1.0};
    const double own_de = side == 0 ? da : db;
    const double sign1 = side == 0 ? 1.0 : -1.0;
    double *other = side == 0 ? up : lo;
    for (int q = 0; q < 4; q++) {
      const double r1 = sign1 * (F[q] - pen * J[q]) / own_de;
      const double r2 = 3.0 * (F[q] + (t / own_de - pen) * J[q]) / own_de;
      // q = 0, 1 act on group a, q = 2, 3 on group b
      const bool on_self = (side == 0) == (q < 2);
      double *blk = on_self ? dd : other;
      blk[0 * 2 + (q & 1)] += r1;
      blk[1 * 2 + (q & 1)] += r2;
    }
  }
}

// Gershgorin bound of the explicit straggling update: a substep of length
// h applies rho h (St / 2) psi explicitly; forward Euler on this operator
// (real, non-positive spectrum) is stable for h rho lambda_max / 2 <= 2.
double strag_row_bound(const pbs_ctx *c) {
  double m = 0.0;
  for (int g = 0; g < c->ng; g++) {
    double b[12];
    strag_blocks(c, g, b);
    for (int r = 0; r < 2; r++) {
      double s = 0.0;
      for (int blk = 0; blk < 3; blk++) s += std::fabs(b[4 * blk + 2 * r]) + std::fabs(b[4 * blk + 2 * r + 1]);
      m = std::max(m, s);
    }
  }
  return m;
}

// Column weights of the deposited energy for the CN straggling step: with
// A the energy operator per unit rho c and phi_g = (E_g dE_g, dE_g^2 / 6),
// Om_g = A_gg^T phi_g + A_{g-1,up}^T phi_{g-1} + A_{g+1,lo}^T phi_{g+1}, so that
// phi^T c A y = rho c sum_g Om_g . y_g.
void omega_table(const pbs_ctx *c, std::vector<double> &om) {
  const int G = c->ng;
  om.assign(2 * (size_t)G, 0.0);
  auto phi = [&](int g, int r) { return r == 0 ? c->e_c[g] * c->de[g] : c->de[g] * c->de[g] / 6.0; };
  for (int g = 0; g < G; g++) {
    double b[12], gg[4], up[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    strag_blocks(c, g, b);
    const double sm = c->s_face[g] / c->de[g], sp = c->s_face[g + 1] / c->de[g], sig = c->sig[g];
    gg[0] = -sm - sig + 0.5 * b[4];
    gg[1] = sm + 0.5 * b[5];
    gg[2] = -3.0 * sp + 0.5 * b[6];
    gg[3] = -sp - 2.0 * sm - sig + 0.5 * b[7];
    if (g > 0) {  // row g-1's block on psi_g
      double bm[12];
      strag_blocks(c, g - 1, bm);
      const double spm = c->s_face[g] / c->de[g - 1];
      up[0] = spm + 0.5 * bm[8];
      up[1] = -spm + 0.5 * bm[9];
      up[2] = 3.0 * spm + 0.5 * bm[10];
      up[3] = -3.0 * spm + 0.5 * bm[11];
    }
    if (g + 1 < G) {  // row g+1's block on psi_g
      double bp[12];
      strag_blocks(c, g + 1, bp);
      for (int i = 0; i < 4; i++) lo[i] = 0.5 * bp[i];
    }
    for (int q = 0; q < 2; q++) {
      double w = 0.0;
      for (int r = 0; r < 2; r++) {
        w += gg[2 * r + q] * phi(g, r);
        if (g > 0) w += up[2 * r + q] * phi(g - 1, r);
        if (g + 1 < G) w += lo[2 * r + q] * phi(g + 1, r);
      }
      om[2 * g + q] = w;
    }
  }
}

// Exponential energy transfer P^1(g' -> g) = lambda e^{-lambda (E_g' - E_g)},
// normalised per emitting group g', and the source weights of the fused
// recursion (q1 = lambda sigma_g' dE_g' / Z_g', decay = e^{-lambda (E_g+1 - E_g)}),
// from the removal cross sections already in c->sig.
void transfer_tables(pbs_ctx *c, double lambda) {
  const int G = c->ng;
  c->p1.assign((size_t)G * G, 0.0);
  c->q1.assign(G, 0.0);
  c->decay.assign(G, 0.0);
  for (int gp = 0; gp < G; gp++) {
    double z = 0.0;
    for (int g = gp; g >= 0; g--) z += lambda * std::exp(-lambda * (c->e_c[gp] - c->e_c[g]));
    for (int g = 0; g <= gp; g++) c->p1[(size_t)gp * G + g] = lambda * std::exp(-lambda * (c->e_c[gp] - c->e_c[g])) / z;
    c->q1[gp] = lambda * c->sig[gp] * c->de[gp] / z;
    c->decay[gp] = (gp + 1 < G) ? std::exp(-lambda * (c->e_c[gp + 1] - c->e_c[gp])) : 0.0;
  }
}

void build_tables(pbs_ctx *c, const pbs_physics &ph) {
  const int G = c->ng, na = c->na;
  c->ts.assign(G, 0.0);
  c->sig.assign(G, ph.sigma_ct);
  // a face at E <= 0 takes the stopping power at half the lowest group width
  // (the Bethe-Bloch tables: at no less than 0.5 MeV)
  const bool bethe = ph.model == 1;
  const double floor_e = bethe ? std::max(0.5 * c->de[0], 0.5) : 0.5 * c->de[0];
  c->s_base.assign(G + 1, 0.0);
  c->t_face.assign(G + 1, 0.0);
  for (int f = 0; f <= G; f++) {
    const double e = std::max(c->e_faces[f], floor_e);
    c->s_base[f] = bethe ? stopping_bethe_water(ph, e) : stopping_bk(ph, e);
    // the straggling formula is held below 0.5 MeV (its logarithm turns
    // negative at a few tens of keV)
    if (ph.t_scale > 0.0) c->t_face[f] = ph.t_scale * straggling_williams_water(ph, std::max(e, 0.5));
  }
  fold_straggling(c);
  // 8-point Gauss-Legendre nodes / weights on [-1, 1] (positive half)
  static const double gl_x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  static const double gl_w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  for (int g = 0; g < G; g++) {
    const double lo = std::max(c->e_faces[g], floor_e), hi = c->e_faces[g + 1];
    if (bethe) {
      const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
      double acc = 0.0;
      for (int q = 0; q < 4; q++)
        acc += gl_w[q] * (scattering_rutherford_water(ph, mid - half * gl_x[q]) +
                          scattering_rutherford_water(ph, mid + half * gl_x[q]));
      c->ts[g] = ph.ts_scale * 0.5 * acc;
    } else {
      c->ts[g] = ph.ts_scale * (highland_primitive(ph, hi) - highland_primitive(ph, lo)) / (hi - lo);
    }
  }
  transfer_tables(c, ph.lambda_p1);
  // angular transfer: Gamma density of the angle between (1,u',v') and (1,u,v),
  // normalised so that sum_a P2 du dv = 1 for every incoming a'
  // (the same [a][a'] block for every group: built once, then copied G times)
  std::vector<double> blk((size_t)na * na), col(na);
  for (int ap = 0; ap < na; ap++) {
    const double u1 = c->u[ap % c->nu], v1 = c->v[ap / c->nu];
    double k = 0.0;
    for (int a = 0; a < na; a++) {
      const double u2 = c->u[a % c->nu], v2 = c->v[a / c->nu];
      const double cx = u2 * v1 - v2 * u1, cy = v2 - v1, cz = u1 - u2;  // (1,u2,v2) x (1,u1,v1)
      const double th = std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), 1.0 + u1 * u2 + v1 * v2);
      col[a] = gamma_density(th, ph.g_alpha, ph.g_beta);
      k += col[a];
    }
    k *= c->du * c->dv;
    for (int a = 0; a < na; a++) blk[(size_t)a * na + ap] = k > 0.0 ? col[a] / k : 0.0;
  }
  c->p2.clear();
  c->p2.reserve((size_t)G * na * na);
  for (int g = 0; g < G; g++) c->p2.insert(c->p2.end(), blk.begin(), blk.end());
}

template <typename st>
st to_storage(double x) { return (st)x; }
template <>
__nv_bfloat16 to_storage<__nv_bfloat16>(double x) { return __float2bfloat16_rn((float)x); }

template <typename st>
double from_storage(st x) { return (double)x; }
template <>
double from_storage<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename real, typename st>
pbs_status upload_tables(pbs_ctx *c) {
  const int G = c->ng;
  std::vector<GroupCoef<real>> coef(G);
  for (int g = 0; g < G; g++) {
    GroupCoef<real> &k = coef[g];
    k.sm = (real)(c->s_face[g] / c->de[g]);
    k.sp = (real)(c->s_face[g + 1] / c->de[g]);
    k.sig = (real)c->sig[g];
    k.ehat = (real)(c->e_c[g] * c->de[g]);
    k.dq = (real)(c->de[g] * c->de[g] / 6.0);
    k.de = (real)c->de[g];
    k.inv_de = (real)(1.0 / c->de[g]);
    k.q1 = (real)c->q1[g];
    k.decay = (real)c->decay[g];
    k.pad = 0;
  }
  std::vector<StragCoef<real>> sc(c->strag ? G : 0);
  for (int g = 0; g < (int)sc.size(); g++) {
    double b[12];
    strag_blocks(c, g, b);
    real *o = reinterpret_cast<real *>(&sc[g]);
    for (int i = 0; i < 12; i++) o[i] = (real)b[i];
  }
  std::vector<real> om_r;
  if (!sc.empty()) {
    PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_strag), sc.data(), sizeof(StragCoef<real>) * G,
                                cudaMemcpyHostToDevice, c->stream));
    std::vector<double> om;
    omega_table(c, om);
    om_r.assign(om.begin(), om.end());
    PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_omega), om_r.data(), sizeof(real) * om_r.size(),
                                cudaMemcpyHostToDevice, c->stream));
  }
  std::vector<real> ts(G);
  for (int g = 0; g < G; g++) ts[g] = (real)c->ts[g];
  PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_coef), coef.data(), sizeof(GroupCoef<real>) * G,
                              cudaMemcpyHostToDevice, c->stream));
  PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_ts), ts.data(), sizeof(real) * G, cudaMemcpyHostToDevice, c->stream));
  std::vector<st> p2;
  if (c->K > 0) {
    p2.resize(c->p2.size());
    for (size_t e = 0; e < p2.size(); e++) p2[e] = to_storage<st>(c->p2[e]);
    PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_p2), p2.data(), sizeof(st) * p2.size(), cudaMemcpyHostToDevice,
                                c->stream));
  }
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));  // host staging buffers die here
  return PBS_OK;
}

// ---------------------------------------------------------------- beam

double std_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// mass of N(mu, s^2) in [lo, hi], evaluated on the tail side for accuracy
double normal_mass(double lo, double hi, double mu, double s) {
  const double a = (lo - mu) / s, b = (hi - mu) / s;
  if (a > 0.0) return std_cdf(-a) - std_cdf(-b);
  return std_cdf(b) - std_cdf(a);
}

void beam_factors(const pbs_ctx *c, const pbs_beam &b, std::vector<double> &out) {
  const int G = c->ng, na = c->na;
  out.assign(2 * G + na + c->ny + c->nz, 0.0);
  double *fe = out.data(), *fa = fe + 2 * G, *fy = fa + na, *fz = fy + c->ny;
  const double inv_sqrt_2pi = 0.3989422804014326779;
  double ne = 0.0, nang = 0.0, nyy = 0.0, nzz = 0.0;
  for (int g = 0; g < G; g++) {
    const double lo = c->e_faces[g], hi = c->e_faces[g + 1], de = c->de[g];
    const double m0 = normal_mass(lo, hi, b.e0, b.sigma_e);
    const double za = (lo - b.e0) / b.sigma_e, zb = (hi - b.e0) / b.sigma_e;
    // int (E - E_g) N(E) dE = s (n(za) - n(zb)) + (E0 - E_g) m0
    const double m1 = b.sigma_e * inv_sqrt_2pi * (std::exp(-0.5 * za * za) - std::exp(-0.5 * zb * zb)) +
                      (b.e0 - c->e_c[g]) * m0;
    fe[2 * g] = m0 / de;                  // (1/dE) int N
    fe[2 * g + 1] = 6.0 * m1 / (de * de); // (3/dE) int N phi^2, phi^2 = 2 (E - E_g)/dE
    ne += fe[2 * g] * de;
  }
  for (int j = 0; j < c->nv; j++)
    for (int i = 0; i < c->nu; i++) {
      const double pu = normal_mass(c->u[i] - 0.5 * c->du, c->u[i] + 0.5 * c->du, b.u0, b.sigma_u) / c->du;
      const double pv = normal_mass(c->v[j] - 0.5 * c->dv, c->v[j] + 0.5 * c->dv, b.v0, b.sigma_v) / c->dv;
      fa[j * c->nu + i] = pu * pv;
      nang += pu * pv * c->du * c->dv;
    }
  // rows of the whole grid (a lateral part projects its rows of it, with the
  // whole grid's normalisation, so that it holds exactly the whole grid's values)
  const int nyg = c->part ? c->part_nyg : c->ny, y0 = c->part ? c->part_y0 : 0;
  for (int pg = 0; pg < nyg; pg++) {
    const double f = normal_mass((pg - 0.5 * nyg) * c->dy, (pg + 1 - 0.5 * nyg) * c->dy, b.y0, b.sigma_y) / c->dy;
    if (pg >= y0 && pg < y0 + c->ny) fy[pg - y0] = f;
    nyy += f * c->dy;
  }
  for (int q = 0; q < c->nz; q++) {
    fz[q] = normal_mass((q - 0.5 * c->nz) * c->dz, (q + 1 - 0.5 * c->nz) * c->dz, b.z0, b.sigma_z) / c->dz;
    nzz += fz[q] * c->dz;
  }
  const double norm = 1.0 / (ne * nang * nyy * nzz);
  for (int e = 0; e < 2 * G; e++) fe[e] *= norm;
}

// ---------------------------------------------------------------- march

// E substeps on the components of beams b0 .. b1-1 in lock-step.  slab_b < 0:
// one substep E(h) with slab_a.  slab_b >= 0: two back-to-back substeps E(h)
// (slab_a, then slab_b) fused in one pass per component.  Fluence after the
// first substep goes to plane flu_plane (if >= 0).
template <typename real, typename st>
pbs_status energy_cn_run(pbs_ctx *c, double h, int slab, int flu_plane, int b0, int b1);

template <typename real, typename st>
pbs_status energy_run(pbs_ctx *c, double h, int slab_a, int slab_b, int flu_plane, int b0, int b1) {
  if (b1 <= b0) return PBS_OK;
  if (c->strag && c->opts.straggling_integrator == 1) {  // no fused pair: two substeps in turn
    pbs_status r = energy_cn_run<real, st>(c, h, slab_a, flu_plane, b0, b1);
    if (r == PBS_OK && slab_b >= 0) r = energy_cn_run<real, st>(c, h, slab_b, -1, b0, b1);
    return r;
  }
  LaunchCtx lc = lctx(c);
  const Dims d = dims_for(c, b1 - b0);
  const size_t nyz = (size_t)c->ny * c->nz;
  const size_t nsrc = (size_t)c->ng * c->na * nyz;
  const size_t half_stride = (size_t)c->B * nsrc;  // second half of a fused pair
  const BeamStrides bs{(long long)(c->K + 1) * c->d.comp_elems, (long long)nsrc, (long long)c->nx * (long long)nyz,
                       (long long)(c->nx + 1) * (long long)nyz};
  real *psi = at<real>(c, c->off_psi) + (size_t)b0 * bs.psi;
  const real *rho = at<real>(c, c->off_rho);
  double *dose = at<double>(c, c->off_dose) + (size_t)b0 * bs.dose;
  double *flu = flu_plane >= 0 ? at<double>(c, c->off_flu) + (size_t)b0 * bs.flu + (size_t)flu_plane * nyz : nullptr;
  st *rbuf = at<st>(c, c->off_r) + (size_t)b0 * nsrc, *sbuf = at<st>(c, c->off_s) + (size_t)b0 * nsrc;
  const auto *coef = at<GroupCoef<real>>(c, c->off_coef);
  const bool two = slab_b >= 0;
  for (int k = 0; k <= c->K; k++) {
    EnergyHalf<real, st> ha{rho + (size_t)slab_a * nyz, (real)(0.5 * h), k >= 1 ? sbuf : nullptr,
                            k < c->K ? rbuf : nullptr, dose + (size_t)slab_a * nyz};
    EnergyHalf<real, st> hb{two ? rho + (size_t)slab_b * nyz : nullptr, (real)(0.5 * h),
                            k >= 1 ? sbuf + half_stride : nullptr, k < c->K ? rbuf + half_stride : nullptr,
                            two ? dose + (size_t)slab_b * nyz : nullptr};
    cudaError_t e;
    {
      ProfScope ps(c, PBS_KERNEL_ENERGY);
      e = launch_energy<real, st>(lc, d, psi + (size_t)k * c->d.comp_elems, ha, two ? &hb : nullptr, coef, flu,
                                  c->du * c->dv / c->dx, c->du * c->dv, bs,
                                  c->strag ? at<StragCoef<real>>(c, c->off_strag) : nullptr);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "energy kernel");
    if (k < c->K) {
      for (int half = 0; half < (two ? 2 : 1); half++) {
        ProfScope ps(c, PBS_KERNEL_SOURCE);
        e = launch_source<real, st>(lc, d, at<st>(c, c->off_p2), rbuf + half * half_stride,
                                    sbuf + half * half_stride, c->du * c->dv, b1 - b0);
        if (e != cudaSuccess) return cuda_fail(c, e, "source kernel");
      }
    }
  }
  return PBS_OK;
}

// One E substep with straggling inside the Crank-Nicolson step (block
// elimination, k_energy_cn.cu): the eliminated blocks of the slab, then per
// component the two passes (and the R recursion), then the source of the
// next component as in energy_run.
template <typename real, typename st>
pbs_status energy_cn_run(pbs_ctx *c, double h, int slab, int flu_plane, int b0, int b1) {
  LaunchCtx lc = lctx(c);
  const Dims d = dims_for(c, b1 - b0);
  const size_t nyz = (size_t)c->ny * c->nz;
  const size_t nsrc = (size_t)c->ng * c->na * nyz;
  const BeamStrides bs{(long long)(c->K + 1) * c->d.comp_elems, (long long)nsrc, (long long)c->nx * (long long)nyz,
                       (long long)(c->nx + 1) * (long long)nyz};
  real *psi = at<real>(c, c->off_psi) + (size_t)b0 * bs.psi;
  const real *rho = at<real>(c, c->off_rho) + (size_t)slab * nyz;
  double *dose = at<double>(c, c->off_dose) + (size_t)b0 * bs.dose + (size_t)slab * nyz;
  double *flu = flu_plane >= 0 ? at<double>(c, c->off_flu) + (size_t)b0 * bs.flu + (size_t)flu_plane * nyz : nullptr;
  st *rbuf = at<st>(c, c->off_r) + (size_t)b0 * nsrc, *sbuf = at<st>(c, c->off_s) + (size_t)b0 * nsrc;
  const auto *coef = at<GroupCoef<real>>(c, c->off_coef);
  const auto *strag = at<StragCoef<real>>(c, c->off_strag);
  real *dinv = at<real>(c, c->off_dinv);
  cudaError_t e;
  {
    ProfScope ps(c, PBS_KERNEL_ENERGY);
    e = launch_cn_factor<real>(lc, d, rho, coef, strag, (real)(0.5 * h), dinv);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "energy factor kernel");
  for (int k = 0; k <= c->K; k++) {
    EnergyHalf<real, st> hs{rho, (real)(0.5 * h), k >= 1 ? sbuf : nullptr, k < c->K ? rbuf : nullptr, dose};
    {
      ProfScope ps(c, PBS_KERNEL_ENERGY);
      e = launch_energy_cn<real, st>(lc, d, psi + (size_t)k * c->d.comp_elems, hs, coef, strag,
                                     at<real>(c, c->off_omega), dinv, flu, c->du * c->dv / c->dx, c->du * c->dv, bs);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "energy kernel");
    if (k < c->K) {
      ProfScope ps(c, PBS_KERNEL_SOURCE);
      e = launch_source<real, st>(lc, d, at<st>(c, c->off_p2), rbuf, sbuf, c->du * c->dv, b1 - b0);
      if (e != cudaSuccess) return cuda_fail(c, e, "source kernel");
    }
  }
  return PBS_OK;
}

template <typename real, typename st>
pbs_status energy_all(pbs_ctx *c, double h, int slab, int flu_plane) {
  return energy_run<real, st>(c, h, slab, -1, flu_plane, 0, c->B);
}

// T(h) on the components of the first nb beams.
template <typename real>
pbs_status transport_run(pbs_ctx *c, double h, int nb) {
  if (nb <= 0) return PBS_OK;
  const Dims d = dims_for(c, nb);
  ProfScope ps(c, PBS_KERNEL_TRANSPORT);
  cudaError_t e = launch_transport_rows<real>(lctx(c), d, at<real>(c, c->off_psi), h, c->du, c->dv, c->dy, c->dz);
  return e == cudaSuccess ? PBS_OK : cuda_fail(c, e, "transport kernel");
}

template <typename real>
pbs_status transport_all(pbs_ctx *c, double h) {
  return transport_run<real>(c, h, c->B);
}

// A(h) on the components of the first nb beams.
template <typename real>
pbs_status angular_run(pbs_ctx *c, double h, int slab, int nb) {
  if (nb <= 0) return PBS_OK;
  const size_t nyz = (size_t)c->ny * c->nz;
  const Dims d = dims_for(c, nb);
  ProfScope ps(c, PBS_KERNEL_ANGULAR);
  cudaError_t e = launch_angular<real>(lctx(c), d, at<real>(c, c->off_psi),
                                       at<real>(c, c->off_rho) + (size_t)slab * nyz, at<real>(c, c->off_ts), h, c->du,
                                       c->dv);
  return e == cudaSuccess ? PBS_OK : cuda_fail(c, e, "angular kernel");
}

template <typename real>
pbs_status angular_all(pbs_ctx *c, double h, int slab) {
  return angular_run<real>(c, h, slab, c->B);
}

// Apply a deferred closing E(h/2) (of depth step steps_done - 1) to the beams
// that marched that step.
template <typename real, typename st>
pbs_status flush_impl(pbs_ctx *c) {
  if (!c->pending) return PBS_OK;
  c->pending = false;
  const int s = c->steps_done - 1;
  return energy_run<real, st>(c, 0.5 * c->dx, s, -1, s + 1, 0, active_at(c, s));
}

// Depth steps.  The closing E(h/2) of a step is deferred and fused with the
// opening E(h/2) of the next (same arithmetic, one pass over psi instead of
// two); any read or substep call applies a deferred half first.  Beams whose
// depth ends at step s - 1 get the closing half alone.
// The four stages of depth step s = steps_done, with act beams marching it:
//   0  E(h/2) opening step s (fused with the deferred closing half of s-1)
//   1  T(h/2)      2  A(h)      3  T(h/2), then the closing half is deferred
// A lateral part of a decomposed beam needs fresh halo rows before stages 1
// and 3; every other stage is local to each lateral point.
template <typename real, typename st>
pbs_status stage_impl(pbs_ctx *c, int stage) {
  const int s = c->steps_done;
  const int act = active_at(c, s);
  pbs_status r = PBS_OK;
  switch (stage) {
    case 0:
      if (c->pending) {
        const int prev = active_at(c, s - 1);
        r = energy_run<real, st>(c, 0.5 * c->dx, s - 1, s, s, 0, act);  // close step s-1, open step s
        if (r == PBS_OK) r = energy_run<real, st>(c, 0.5 * c->dx, s - 1, -1, s, act, prev);  // close only
      } else {
        r = energy_run<real, st>(c, 0.5 * c->dx, s, -1, -1, 0, act);
      }
      c->pending = false;
      return r;
    case 1:
      return transport_run<real>(c, 0.5 * c->dx, act);
    case 2:
      return angular_run<real>(c, c->dx, s, act);
    default:
      if ((r = transport_run<real>(c, 0.5 * c->dx, act)) != PBS_OK) return r;
      c->pending = act > 0;
      c->steps_done++;
      return PBS_OK;
  }
}

template <typename real, typename st>
pbs_status step_impl(pbs_ctx *c, int n) {
  for (int i = 0; i < n; i++)
    for (int stage = 0; stage < 4; stage++) {
      pbs_status r = stage_impl<real, st>(c, stage);
      if (r != PBS_OK) return r;
    }
  return PBS_OK;
}

// Halo rows of the lateral parts P[0..n-1] (ordered by row): each interior
// interface copies the rows each side needs from the other's own rows into
// its own workspace, for every (component, group, coefficient, angle) plane:
// two strided copies (cudaMemcpy2DAsync) per interface.  Parts on other
// streams or devices are ordered by event waits before and after the copies,
// so that neither side's next transport overwrites rows still being read.
pbs_status join_streams(pbs_ctx *a, pbs_ctx *b) {
  if (a->stream == b->stream && a->dev == b->dev) return PBS_OK;
  for (pbs_ctx *x : {a, b}) {
    pbs_ctx *y = x == a ? b : a;
    PBS_CUDA(x, cudaSetDevice(x->dev));
    if (!x->xev) PBS_CUDA(x, cudaEventCreateWithFlags(&x->xev, cudaEventDisableTiming));
    PBS_CUDA(x, cudaEventRecord(x->xev, x->stream));
    PBS_CUDA(x, cudaSetDevice(y->dev));
    PBS_CUDA(x, cudaStreamWaitEvent(y->stream, x->xev, 0));
  }
  return PBS_OK;
}

pbs_status copy_rows(pbs_ctx *dst, int dst_row, pbs_ctx *src, int src_row, int rows) {
  if (rows <= 0) return PBS_OK;
  const size_t rs = dst->rsize, row = (size_t)dst->nz * rs;
  const size_t planes = (size_t)dst->d.ncomp * dst->ng * 2 * dst->na;
  unsigned char *d = at<unsigned char>(dst, dst->off_psi) + (size_t)dst_row * row;
  const unsigned char *q = at<unsigned char>(src, src->off_psi) + (size_t)src_row * row;
  const size_t dp = (size_t)dst->ny * row, sp = (size_t)src->ny * row;
  PBS_CUDA(dst, cudaSetDevice(dst->dev));
  for (size_t p0 = 0; p0 < planes; p0 += 32768) {  // in chunks of planes
    const size_t np = std::min<size_t>(32768, planes - p0);
    PBS_CUDA(dst, cudaMemcpy2DAsync(d + p0 * dp, dp, q + p0 * sp, sp, (size_t)rows * row, np, cudaMemcpyDefault,
                                    dst->stream));
  }
  return PBS_OK;
}

pbs_status exchange_halos(pbs_ctx *const *P, int n) {
  for (int i = 0; i + 1 < n; i++) {
    pbs_ctx *lo = P[i], *hi = P[i + 1];
    pbs_status r = join_streams(lo, hi);
    if (r != PBS_OK) return r;
    // lo's upper halo <- hi's rows; hi's lower halo <- lo's rows
    const int lo_halo_g = lo->part_y0 + lo->ny - lo->halo_hi;  // first global row of lo's upper halo
    if ((r = copy_rows(lo, lo->ny - lo->halo_hi, hi, lo_halo_g - hi->part_y0, lo->halo_hi)) != PBS_OK) return r;
    if ((r = copy_rows(hi, 0, lo, hi->part_y0 - lo->part_y0, hi->halo_lo)) != PBS_OK) return r;
    if ((r = join_streams(lo, hi)) != PBS_OK) return r;
  }
  return PBS_OK;
}

template <typename real, typename st>
pbs_status domain_step_impl(pbs_ctx *const *P, int n, int n_steps) {
  int dev0 = 0;
  cudaGetDevice(&dev0);
  pbs_status r = PBS_OK;
  for (int i = 0; i < n_steps && r == PBS_OK; i++)
    for (int stage = 0; stage < 4 && r == PBS_OK; stage++) {
      if (stage == 1 || stage == 3) r = exchange_halos(P, n);
      for (int j = 0; j < n && r == PBS_OK; j++) {
        if (cudaSetDevice(P[j]->dev) != cudaSuccess) r = fail(P[j], PBS_ERR_CUDA, "cudaSetDevice");
        else r = stage_impl<real, st>(P[j], stage);
      }
    }
  cudaSetDevice(dev0);
  return r;
}

// Restart every beam from its projection (factors already on the device):
// zero psi, dose, fluence and the status word, project, tally plane 0.
// Device work only, so it can be captured into a graph.
template <typename real, typename st>
pbs_status reinit_impl(pbs_ctx *c) {
  const size_t nyz = (size_t)c->ny * c->nz;
  // the projection overwrites every primary component; only scattered ones need zeroing
  if (c->K > 0)
    PBS_CUDA(c, cudaMemsetAsync(at<void>(c, c->off_psi), 0, (size_t)c->d.ncomp * c->d.comp_elems * sizeof(real),
                                c->stream));
  PBS_CUDA(c, cudaMemsetAsync(at<void>(c, c->off_dose), 0, (size_t)c->B * c->nx * nyz * 8, c->stream));
  PBS_CUDA(c, cudaMemsetAsync(at<void>(c, c->off_flu), 0, (size_t)c->B * (c->nx + 1) * nyz * 8, c->stream));
  PBS_CUDA(c, cudaMemsetAsync(at<void>(c, c->off_err), 0, 64, c->stream));
  const Dims d1 = dims_for(c, 1);
  for (int b = 0; b < c->B; b++) {
    const double *fe = at<double>(c, c->off_init) + (size_t)b * init_stride(c);
    real *psi_b = at<real>(c, c->off_psi) + (size_t)b * (c->K + 1) * c->d.comp_elems;
    cudaError_t e = launch_init<real>(lctx(c), d1, psi_b, fe, fe + 2 * c->ng, fe + 2 * c->ng + c->na,
                                      fe + 2 * c->ng + c->na + c->ny);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    e = launch_fluence<real>(lctx(c), d1, psi_b, c->K + 1, at<GroupCoef<real>>(c, c->off_coef),
                             at<double>(c, c->off_flu) + (size_t)b * (c->nx + 1) * nyz, c->du * c->dv);
    if (e != cudaSuccess) return cuda_fail(c, e, "fluence kernel");
  }
  c->steps_done = 0;
  c->pending = false;
  c->stage = 0;
  return PBS_OK;
}

template <typename real, typename st>
pbs_status launch_impl(pbs_ctx *c, const pbs_beam *beams) {
  std::vector<double> f((size_t)c->B * init_stride(c)), one;
  for (int b = 0; b < c->B; b++) {
    beam_factors(c, beams[b], one);
    std::copy(one.begin(), one.end(), f.begin() + (size_t)b * init_stride(c));
  }
  PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, c->off_init), f.data(), f.size() * 8, cudaMemcpyHostToDevice, c->stream));
  pbs_status r = reinit_impl<real, st>(c);
  if (r != PBS_OK) return r;
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));  // f dies here
  return PBS_OK;
}

// The whole march of every beam (restart, steps to the deepest beam's depth,
// closing half), issued on the context's stream.
template <typename real, typename st>
pbs_status run_impl(pbs_ctx *c) {
  pbs_status r = reinit_impl<real, st>(c);
  if (r != PBS_OK) return r;
  if ((r = step_impl<real, st>(c, max_depth(c))) != PBS_OK) return r;
  return flush_impl<real, st>(c);
}

// Record run_impl into a CUDA graph on a private stream (once per beam
// depths / material extent / launch shapes) and launch it on the context's
// stream.
template <typename real, typename st>
pbs_status run_graph_impl(pbs_ctx *c) {
  const int depth = max_depth(c);
  if (!c->graph || c->graph_depth != depth) {
    drop_graph(c);
    if (!c->cap_stream) PBS_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    const long long before = c->launches;
    c->stream = c->cap_stream;
    c->capturing = true;
    cudaGraph_t g = nullptr;
    pbs_status r = PBS_OK;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      r = run_impl<real, st>(c);
      cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    c->capturing = false;
    c->graph_kernels = c->launches - before;  // kernels per replay, counted when they run
    c->launches = before;
    if (r != PBS_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return cuda_fail(c, e, "graph instantiate");
    }
    c->graph_depth = depth;
  }
  PBS_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
  c->launches += c->graph_kernels;
  c->steps_done = depth;
  c->pending = false;
  return PBS_OK;
}

pbs_status check_device_status(pbs_ctx *c) {
  int w[2] = {0, 0};
  PBS_CUDA(c, cudaMemcpyAsync(w, at<void>(c, c->off_err), sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  if (w[0] != 0) return fail(c, PBS_ERR_TIMEOUT, "a device wait gave up (code " + std::to_string(w[1]) + ")");
  return PBS_OK;
}

template <typename real>
pbs_status read_psi_impl(pbs_ctx *c, int k, double *out) {
  std::vector<real> tmp(c->d.comp_elems);
  PBS_CUDA(c, cudaMemcpyAsync(tmp.data(), at<real>(c, c->off_psi) + (size_t)k * c->d.comp_elems,
                              sizeof(real) * tmp.size(), cudaMemcpyDeviceToHost, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t e = 0; e < tmp.size(); e++) out[e] = (double)tmp[e];
  return check_device_status(c);
}

template <typename real>
pbs_status write_psi_impl(pbs_ctx *c, int k, const double *in) {
  std::vector<real> tmp(c->d.comp_elems);
  for (size_t e = 0; e < tmp.size(); e++) tmp[e] = (real)in[e];
  PBS_CUDA(c, cudaMemcpyAsync(at<real>(c, c->off_psi) + (size_t)k * c->d.comp_elems, tmp.data(),
                              sizeof(real) * tmp.size(), cudaMemcpyHostToDevice, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return PBS_OK;
}

template <typename real>
pbs_status set_material_impl(pbs_ctx *c, const double *rho, int n) {
  const size_t cnt = (size_t)n * c->ny * c->nz;
  std::vector<real> tmp(cnt);
  for (size_t e = 0; e < cnt; e++) tmp[e] = (real)rho[e];
  PBS_CUDA(c, cudaMemcpyAsync(at<real>(c, c->off_rho), tmp.data(), sizeof(real) * cnt, cudaMemcpyHostToDevice,
                              c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return PBS_OK;
}

template <typename real, typename st>
pbs_status eval_source_impl(pbs_ctx *c, int k_from, int slab, double *out) {
  const size_t nyz = (size_t)c->ny * c->nz;
  cudaError_t e = launch_source_input(lctx(c), c->d, at<real>(c, c->off_psi) + (size_t)k_from * c->d.comp_elems,
                                      at<real>(c, c->off_rho) + (size_t)slab * nyz, at<void>(c, c->off_coef),
                                      at<void>(c, c->off_r), c->precision);
  if (e != cudaSuccess) return cuda_fail(c, e, "source input kernel");
  e = launch_source<real, st>(lctx(c), c->d, at<st>(c, c->off_p2), at<st>(c, c->off_r), at<st>(c, c->off_s),
                              c->du * c->dv);
  if (e != cudaSuccess) return cuda_fail(c, e, "source kernel");
  const size_t n = (size_t)c->ng * c->na * nyz;
  std::vector<st> tmp(n);
  PBS_CUDA(c, cudaMemcpyAsync(tmp.data(), at<st>(c, c->off_s), sizeof(st) * n, cudaMemcpyDeviceToHost, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < n; i++) out[i] = from_storage<st>(tmp[i]);
  return PBS_OK;
}

bool ready_to_march(pbs_ctx *c) { return c->ws && c->have_tables && c->have_material && c->have_beam; }

// Explicit straggling is stable while a substep h keeps
// h rho_max lambda_max(St) / 2 <= 2 (Gershgorin bound of lambda_max).
pbs_status strag_guard(pbs_ctx *c, double h) {
  if (!c->strag || c->opts.straggling_integrator == 1) return PBS_OK;  // CN: no bound
  if (h * c->rho_max * c->strag_bound > 4.0)
    return fail(c, PBS_ERR_ARG,
                "explicit straggling unstable for this step: h rho T / dE^2 too large (refine dx or coarsen the groups)");
  return PBS_OK;
}

// Launch-shape autotuner.  Times each candidate shape of the energy pass
// (angles per block) and of the streaming transport (resident CTAs per SM)
// on the launched beams with CUDA events, best of `reps`, keeps the fastest,
// then restarts the beams from their projections (the trial passes advance
// the state).  Every candidate computes the same psi; only the summation
// order of the dose reduction depends on the energy shape.
template <typename real, typename st>
pbs_status autotune_impl(pbs_ctx *c, int reps) {
  pbs_status r = flush_impl<real, st>(c);
  if (r != PBS_OK) return r;
  const bool prof = c->profiling;
  c->profiling = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PBS_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, PBS_ERR_CUDA, "event create");
  }
  auto time_best = [&](auto &&fn, float &best) -> pbs_status {
    best = 1e30f;
    for (int i = 0; i < reps; i++) {
      PBS_CUDA(c, cudaEventRecord(e0, c->stream));
      pbs_status q = fn();
      if (q != PBS_OK) return q;
      PBS_CUDA(c, cudaEventRecord(e1, c->stream));
      PBS_CUDA(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      PBS_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    return PBS_OK;
  };
  const int slab_b = c->n_slabs > 1 ? 1 : 0;
  pbs_tuning pick = c->tune;
  float best = 1e30f;
  for (int form : {1, 0}) {
    if (form == 1 && sizeof(real) != 4) continue;
    for (int ay : {4, 8, 16}) {
      c->tune.energy_form = form;
      c->tune.energy_angles = ay;
      float ms;
      r = time_best([&] { return energy_run<real, st>(c, 0.5 * c->dx, 0, slab_b, -1, 0, c->B); }, ms);
      if (r != PBS_OK) break;
      if (ms < best) { best = ms; pick.energy_form = form; pick.energy_angles = ay; }
    }
    if (r != PBS_OK) break;
  }
  c->tune = pick;
  best = 1e30f;
  if (r == PBS_OK) {
    for (int cols : {4, 6, 8}) {
      if (c->nz % cols != 0) continue;
      for (int ctas : {1, 2, 3, 4, 0}) {
        c->tune.transport_cols = cols;
        c->tune.transport_ctas = ctas;
        float ms;
        r = time_best([&] { return transport_run<real>(c, 0.5 * c->dx, c->B); }, ms);
        if (r != PBS_OK) break;
        if (ms < best) { best = ms; pick.transport_ctas = ctas; pick.transport_cols = cols; }
      }
      if (r != PBS_OK) break;
    }
  }
  c->tune = pick;
  best = 1e30f;
  if (r == PBS_OK) {
    for (int form : {5, 7, 6, 2, 3, 4, 1, 0}) {
      c->tune.angular_form = form;
      float ms;
      r = time_best([&] { return angular_run<real>(c, c->dx, 0, c->B); }, ms);
      if (r != PBS_OK) break;
      if (ms < best) { best = ms; pick.angular_form = form; }
    }
  }
  c->tune = pick;
  best = 1e30f;
  if (r == PBS_OK && c->K > 0 && c->precision == PBS_MIXED) {
    for (int form : {2, 1, 0}) {
      c->tune.source_form = form;
      float ms;
      r = time_best([&] {
        cudaError_t e = launch_source<real, st>(lctx(c), dims_for(c, c->B), at<st>(c, c->off_p2), at<st>(c, c->off_r),
                                                at<st>(c, c->off_s), c->du * c->dv, c->B);
        return e == cudaSuccess ? PBS_OK : cuda_fail(c, e, "source kernel");
      }, ms);
      if (r != PBS_OK) break;
      if (ms < best) { best = ms; pick.source_form = form; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->profiling = prof;
  c->tune = pick;
  drop_graph(c);
  if (r != PBS_OK) return r;
  if ((r = reinit_impl<real, st>(c)) != PBS_OK) return r;
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return PBS_OK;
}

}  // namespace

// Checkpoint layout: CkptHeader, then psi (ncomp * comp_elems * rsize), dose
// (B * nx * nyz doubles), fluence (B * (nx + 1) * nyz doubles), beam factors
// (B * init_stride doubles), beam depth ranges (B ints).  The header also
// records what the saved state was marched with but does not contain: the
// method options, a hash of the FP64 host tables and of the density field;
// a restore into a context that differs in any of them is refused.
struct CkptHeader {
  char magic[8];
  int version, precision, ny, nz, ng, nu, nv, nx, K, B, steps_done, pending, have_beam, n_slabs_at_save;
  int angular_integrator, transport_integrator, straggling_integrator, pad;
  unsigned long long tables_hash, material_hash;
};

namespace {
// FNV-1a with 64-bit words in place of bytes (the tables are doubles; a
// consistency check, not a cryptographic one), continuing from h.
unsigned long long fnv1a(unsigned long long h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    unsigned long long w;
    std::memcpy(&w, b + i, 8);
    h ^= w;
    h *= 1099511628211ULL;
  }
  for (; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ULL;
  }
  return h;
}

unsigned long long tables_hash(const pbs_ctx *c) {
  unsigned long long h = 14695981039346656037ULL;
  for (const std::vector<double> *v : {&c->e_faces, &c->s_face, &c->s_base, &c->t_face, &c->ts, &c->sig, &c->p1,
                                       &c->p2, &c->q1, &c->decay})
    h = fnv1a(h, v->data(), v->size() * sizeof(double));
  return h;
}

size_t ckpt_bytes(const pbs_ctx *c) {
  const size_t nyz = (size_t)c->ny * c->nz;
  return sizeof(CkptHeader) + (size_t)c->d.ncomp * c->d.comp_elems * c->rsize + (size_t)c->B * c->nx * nyz * 8 +
         (size_t)c->B * (c->nx + 1) * nyz * 8 + (size_t)c->B * init_stride(c) * 8 + (size_t)c->B * sizeof(int);
}
}  // namespace

namespace {

// ---------------------------------------------------------------- persistent batch

// Slab stacks per chunk of a pipelined transport / angular pass (the
// angular tile's stack count): with pipeline on, the angular step of a chunk
// starts as soon as the first transport of that chunk is done, and the second
// transport of a chunk as soon as its angular step is, so the three passes of
// one beam overlap; without, each pass is one chunk.
constexpr long long kBatchChunk = 32;

struct BatchLayout {
  size_t off_beams, off_tasks, off_queue, off_done, off_next, off_prof, total;
  long long ntasks, nctr;
};

// Depth a beam marches in the batch: its own, or at most max_steps (>= 0)
// for the autotuner's short trials.
int batch_depth(const pbs_ctx *c, int max_steps) {
  const int d = beam_depth(c, 0);
  return max_steps >= 0 ? std::min(d, max_steps) : d;
}

long long batch_chunks(const pbs_ctx *c, int pipeline) {
  const long long nst = (long long)c->d.ncomp * c->ng * 2;
  return pipeline ? (nst + kBatchChunk - 1) / kBatchChunk : 1;
}

BatchLayout batch_layout(pbs_ctx *const *P, int n, int pipeline, int max_steps = -1) {
  BatchLayout L{};
  long long nt = 0, nc = 0;
  for (int i = 0; i < n; i++) {
    const long long steps = batch_depth(P[i], max_steps), nch = batch_chunks(P[i], pipeline);
    nt += steps > 0 ? steps * (1 + 3 * nch) + 1 : 0;  // per step E and, per chunk, T A T; then the closing E
    nc += 2 + 2 * nch;                                // E, T1 per chunk, A per chunk, T2
  }
  L.ntasks = nt;
  L.nctr = nc;
  size_t o = 0;
  L.off_beams = o; o = align256(o + sizeof(BatchBeam) * (size_t)n);
  L.off_tasks = o; o = align256(o + sizeof(BatchTask) * (size_t)nt);
  L.off_queue = o; o = align256(o + sizeof(BatchQueue));
  L.off_done = o; o = align256(o + 8 * (size_t)nc);
  L.off_next = o; o = align256(o + 8 * (size_t)nt);
  L.off_prof = o; o = align256(o + 8 * 8);
  L.total = o;
  return L;
}

// What the persistent kernel handles: FP32 psi (FP32 or mixed precision, no
// scattered component, so the mixed form runs in FP32 too), one beam per
// context, the default integrators, no straggling, even ny*nz, rows a
// multiple of 4 columns, angle grids of at most 8 x 8 shared by the batch,
// all contexts on one device and stream, launched and not mid-step.
pbs_status batch_check(pbs_ctx *const *P, int n, const pbs_batch_options &opt) {
  pbs_ctx *c0 = P[0];
  for (int i = 0; i < n; i++) {
    pbs_ctx *c = P[i];
    if (!ready_to_march(c)) return fail(c0, PBS_ERR_STATE, "every beam needs a workspace, tables, material and a launched beam");
    if (c->stage != 0) return fail(c0, PBS_ERR_STATE, "a staged step is in progress on a beam");
    if (c->precision == PBS_FP64 || c->K != 0 || c->B != 1 || c->strag || c->opts.angular_integrator != 0 ||
        c->opts.transport_integrator != 0 || ((c->ny * c->nz) & 1) || c->nz % 4 != 0 || !batch_supported(c->nu, c->nv))
      return fail(c0, PBS_ERR_UNSUPPORTED,
                  "the persistent batch takes FP32/mixed beams with K = 0, one beam per context, the default "
                  "integrators, no straggling, even ny*nz, nz a multiple of 4 and at most 8 x 8 angles");
    if (c->dev != c0->dev || c->stream != c0->stream)
      return fail(c0, PBS_ERR_ARG, "the beams of a batch share one device and one stream");
    if (c->nu != c0->nu || c->nv != c0->nv || c->u_max != c0->u_max || c->v_max != c0->v_max)
      return fail(c0, PBS_ERR_ARG, "the beams of a batch share one angle grid");
    if (std::max(c->nu, c->nv) > 8 && opt.shape != 0)
      return fail(c0, PBS_ERR_UNSUPPORTED, "16 x 16 angles need batch shape 0");
    for (int j = 0; j < i; j++)
      if (P[j] == c) return fail(c0, PBS_ERR_ARG, "a context appears twice in the batch");
    if (batch_shape(c->d, opt.shape, opt.transport_cols).smem > 160 * 1024)
      return fail(c0, PBS_ERR_UNSUPPORTED, "too many energy groups for the batch");
  }
  return PBS_OK;
}

// Descriptors of the batch (beams, round-robin task list) in host memory.
void batch_descriptors(pbs_ctx *const *P, int n, const BatchLayout &L, const pbs_batch_options &opt, int max_steps,
                       std::vector<BatchBeam> &beams, std::vector<BatchTask> &tasks, size_t &smem) {
  const int hold_beam = opt.hold_beam;
  beams.assign(n, BatchBeam{});
  tasks.clear();
  tasks.reserve((size_t)L.ntasks);
  smem = 0;
  std::vector<BatchShape> shape(n);
  int max_passes = 0;
  for (int b = 0; b < n; b++) {
    pbs_ctx *c = P[b];
    const BatchShape sh = batch_shape(c->d, opt.shape, opt.transport_cols);
    shape[b] = sh;
    smem = std::max(smem, sh.smem);
    BatchBeam &m = beams[b];
    m.psi = at<float>(c, c->off_psi);
    m.rho = at<float>(c, c->off_rho);
    m.coef = at<GroupCoef<float>>(c, c->off_coef);
    m.ts = at<float>(c, c->off_ts);
    m.dose = at<double>(c, c->off_dose);
    m.flu = at<double>(c, c->off_flu);
    m.err = at<int>(c, c->off_err);
    m.d = c->d;
    m.n_steps = batch_depth(c, max_steps);
    // the constants of the per-substep launches, rounded the same way
    const double h = 0.5 * c->dx;
    m.c = (float)(0.5 * h);
    m.hq = (float)(0.25 * c->dx);
    m.ky = (float)(h / c->dy);
    m.kz = (float)(h / c->dz);
    m.du = (float)c->du;
    m.dv = (float)c->dv;
    m.dose_scale = c->du * c->dv / c->dx;
    m.flu_scale = c->du * c->dv;
    m.e_bx = sh.e_bx;
    m.a_bx = sh.a_bx;
    m.tr_kv = sh.tr_kv;
    m.tr_nseg = sh.tr_nseg;
    m.tr_segw = sh.tr_segw;
    m.tr_gw = sh.tr_gw;
    m.tr_stacks = sh.tr_stacks;
    max_passes = std::max(max_passes, m.n_steps);
  }
  (void)max_passes;
  // every beam's own task sequence (each wait names tiles earlier in it),
  // then merged round-robin over the beams, which keeps each beam's order
  std::vector<std::vector<BatchTask>> seq(n);
  int ctr = 0;
  size_t longest = 0;
  for (int b = 0; b < n; b++) {
    const BatchShape &sh = shape[b];
    const long long steps = beams[b].n_steps, nst = sh.tr_stacks, nch = batch_chunks(P[b], opt.pipeline);
    const long long csz = opt.pipeline ? kBatchChunk : nst;
    const int cE = ctr, cT1 = ctr + 1, cA = ctr + 1 + (int)nch, cT2 = ctr + 1 + 2 * (int)nch;
    ctr += 2 + 2 * (int)nch;
    std::vector<long long> t_tiles(nch), a_tiles(nch);
    long long t2tot = 0;
    for (long long c = 0; c < nch; c++) {
      const long long k = std::min(csz, nst - c * csz);
      t_tiles[c] = 2 * k;
      a_tiles[c] = (long long)sh.a_bx * ((k + 31) / 32);
      t2tot += t_tiles[c];
    }
    std::vector<BatchTask> &q = seq[b];
    auto add = [&](int kind, int step, long long first, long long k, long long tiles, int wc, long long need, int sc) {
      q.push_back(BatchTask{b, kind, step, wc, sc, 0, first, k, tiles, need});
    };
    for (long long st = 0; st < steps; st++) {
      if (st == 0) add(kPassEOpen, 0, 0, 0, sh.e_tiles, -1, 0, cE);
      else add(kPassEPair, (int)st, 0, 0, sh.e_tiles, cT2, st * t2tot, cE);
      for (long long i = 0; i < nch + 2; i++) {
        if (i < nch)
          add(kPassT, (int)st, i * csz, t_tiles[i] / 2, t_tiles[i], cE, (st + 1) * sh.e_tiles, cT1 + (int)i);
        if (i >= 1 && i - 1 < nch) {
          const long long c = i - 1;
          add(kPassA, (int)st, c * csz, t_tiles[c] / 2, a_tiles[c], cT1 + (int)c, (st + 1) * t_tiles[c], cA + (int)c);
        }
        if (i >= 2 && i - 2 < nch) {
          const long long c = i - 2;
          add(kPassT, (int)st, c * csz, t_tiles[c] / 2, t_tiles[c], cA + (int)c, (st + 1) * a_tiles[c], cT2);
        }
      }
    }
    if (steps > 0) add(kPassEClose, (int)steps, 0, 0, sh.e_tiles, cT2, steps * t2tot, cE);
    // the test hook: one tile more than can complete, so no wait on it ends
    if (b == hold_beam && q.size() > 1) q[1].wait_need += 1;
    longest = std::max(longest, q.size());
  }
  for (size_t k = 0; k < longest; k++)
    for (int b = 0; b < n; b++)
      if (k < seq[b].size()) tasks.push_back(seq[b][k]);
}

unsigned long long batch_key(pbs_ctx *const *P, int n, void *ws, size_t bytes, long long wait_cycles,
                             const pbs_batch_options &opt, int max_steps) {
  unsigned long long h = 14695981039346656037ULL;
  const int hold = opt.hold_beam;
  h = fnv1a(h, &opt.shape, sizeof(int));
  h = fnv1a(h, &opt.transport_cols, sizeof(int));
  h = fnv1a(h, &opt.pipeline, sizeof(int));
  h = fnv1a(h, &max_steps, sizeof(int));
  for (int i = 0; i < n; i++) {
    const void *ptr = P[i];
    const int depth = beam_depth(P[i], 0);
    h = fnv1a(h, &ptr, sizeof(ptr));
    h = fnv1a(h, &P[i]->ws, sizeof(void *));
    h = fnv1a(h, &depth, sizeof(depth));
  }
  h = fnv1a(h, &n, sizeof(n));
  h = fnv1a(h, &ws, sizeof(ws));
  h = fnv1a(h, &bytes, sizeof(bytes));
  h = fnv1a(h, &wait_cycles, sizeof(wait_cycles));
  h = fnv1a(h, &hold, sizeof(hold));
  return h;
}

// The batch's device work, issued on the lead context's stream: every beam
// restarted from its projection, the queue counters cleared, the
// persistent launch.
pbs_status batch_issue(pbs_ctx *const *P, int n, unsigned char *ws, const BatchLayout &L, long long wait_cycles,
                       size_t smem, int shape) {
  pbs_ctx *c0 = P[0];
  for (int b = 0; b < n; b++) {
    pbs_status r = P[b]->precision == PBS_FP32 ? reinit_impl<float, float>(P[b])
                                               : reinit_impl<float, __nv_bfloat16>(P[b]);
    if (r != PBS_OK) return r;
  }
  PBS_CUDA(c0, cudaMemsetAsync(ws + L.off_queue, 0, L.total - L.off_queue, c0->stream));
  LaunchCtx lc = lctx(c0);
  unsigned long long *prof = c0->profiling ? reinterpret_cast<unsigned long long *>(ws + L.off_prof) : nullptr;
  int ctas = 0;
  cudaError_t e = launch_batch(lc, shape, c0->nu, c0->nv, reinterpret_cast<const BatchBeam *>(ws + L.off_beams), n,
                               reinterpret_cast<const BatchTask *>(ws + L.off_tasks), (int)L.ntasks,
                               reinterpret_cast<BatchQueue *>(ws + L.off_queue),
                               reinterpret_cast<unsigned long long *>(ws + L.off_done),
                               reinterpret_cast<unsigned long long *>(ws + L.off_next), wait_cycles, smem, c0->du,
                               c0->dv, prof, &ctas);
  if (prof && !c0->capturing) {
    c0->batch_prof = prof;
    c0->batch_ctas = ctas;
  }
  return e == cudaSuccess ? PBS_OK : cuda_fail(c0, e, "batch kernel");
}

pbs_status run_batch_impl(pbs_ctx *const *beams, int n_beams, void *dev_ws, size_t bytes,
                          const pbs_batch_options &opt, int max_steps) {
  pbs_ctx *c0 = beams[0];
  if (opt.hold_beam < -1 || opt.hold_beam >= n_beams) return fail(c0, PBS_ERR_ARG, "hold_beam out of range");
  if (opt.shape < 0 || opt.shape > 1 || (opt.transport_cols != 0 && opt.transport_cols != 4 && opt.transport_cols != 6) ||
      opt.pipeline < 0 || opt.pipeline > 1)
    return fail(c0, PBS_ERR_ARG, "batch shape must be 0 or 1, transport_cols 0, 4 or 6, pipeline 0 or 1");
  pbs_status r = batch_check(beams, n_beams, opt);
  if (r != PBS_OK) return r;
  const BatchLayout L = batch_layout(beams, n_beams, opt.pipeline, max_steps);
  if (!dev_ws || bytes < L.total || ((uintptr_t)dev_ws & 255))
    return fail(c0, PBS_ERR_ARG, "batch workspace missing, smaller than pbs_batch_workspace_size or not 256-byte aligned");
  if (L.ntasks > INT_MAX) return fail(c0, PBS_ERR_UNSUPPORTED, "too many passes in the batch");
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c0->dev) != cudaSuccess || khz <= 0) khz = 2000000;
  const double ms = opt.wait_limit_ms > 0 ? opt.wait_limit_ms : 2000.0;
  const long long wait_cycles = (long long)(ms * khz);
  unsigned char *ws = static_cast<unsigned char *>(dev_ws);
  const unsigned long long key = batch_key(beams, n_beams, dev_ws, bytes, wait_cycles, opt, max_steps);
  std::vector<BatchBeam> hb;
  std::vector<BatchTask> ht;
  size_t smem = 0;
  batch_descriptors(beams, n_beams, L, opt, max_steps, hb, ht, smem);
  if (key != c0->batch_key) {  // new batch: upload its descriptors, forget its graph
    PBS_CUDA(c0, batch_init_tables());
    PBS_CUDA(c0, cudaMemcpyAsync(ws + L.off_beams, hb.data(), sizeof(BatchBeam) * hb.size(), cudaMemcpyHostToDevice,
                                 c0->stream));
    if (!ht.empty())
      PBS_CUDA(c0, cudaMemcpyAsync(ws + L.off_tasks, ht.data(), sizeof(BatchTask) * ht.size(), cudaMemcpyHostToDevice,
                                   c0->stream));
    PBS_CUDA(c0, cudaStreamSynchronize(c0->stream));  // the host copies die here
    if (c0->batch_graph) cudaGraphExecDestroy(c0->batch_graph);
    c0->batch_graph = nullptr;
    c0->batch_key = key;
  }
  if (!opt.use_graph) {
    r = batch_issue(beams, n_beams, ws, L, wait_cycles, smem, opt.shape);
    if (r != PBS_OK) return r;
  } else {
    if (!c0->batch_graph) {
      if (!c0->cap_stream) PBS_CUDA(c0, cudaStreamCreateWithFlags(&c0->cap_stream, cudaStreamNonBlocking));
      cudaStream_t user = c0->stream;
      std::vector<long long> before(n_beams);
      for (int b = 0; b < n_beams; b++) {
        before[b] = beams[b]->launches;
        beams[b]->stream = c0->cap_stream;
        beams[b]->capturing = true;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c0->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        r = batch_issue(beams, n_beams, ws, L, wait_cycles, smem, opt.shape);
        cudaError_t e2 = cudaStreamEndCapture(c0->cap_stream, &g);
        if (e == cudaSuccess) e = e2;
      }
      long long kernels = 0;
      for (int b = 0; b < n_beams; b++) {
        beams[b]->stream = user;
        beams[b]->capturing = false;
        kernels += beams[b]->launches - before[b];
        beams[b]->launches = before[b];
      }
      if (r != PBS_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return cuda_fail(c0, e, "batch graph capture");
      e = cudaGraphInstantiate(&c0->batch_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        c0->batch_graph = nullptr;
        return cuda_fail(c0, e, "batch graph instantiate");
      }
      c0->batch_graph_kernels = kernels;
    }
    PBS_CUDA(c0, cudaGraphLaunch(c0->batch_graph, c0->stream));
    c0->launches += c0->batch_graph_kernels;
  }
  for (int b = 0; b < n_beams; b++) {
    beams[b]->steps_done = batch_depth(beams[b], max_steps);
    beams[b]->pending = false;
    beams[b]->stage = 0;
  }
  return PBS_OK;
}

}  // namespace

#define PBS_DISPATCH(c, FN, ...)                                                    \
  ((c)->precision == PBS_FP64    ? FN<double, double>(__VA_ARGS__)                  \
   : (c)->precision == PBS_FP32 ? FN<float, float>(__VA_ARGS__)                     \
                                 : FN<float, __nv_bfloat16>(__VA_ARGS__))
#define PBS_DISPATCH_R(c, FN, ...) \
  ((c)->precision == PBS_FP64 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

extern "C" {

pbs_status pbs_create(pbs_ctx **out, const pbs_grid *g, int precision, void *stream) {
  if (!out || !g || !g->e_faces) return PBS_ERR_ARG;
  *out = nullptr;
  if (g->ny < 1 || g->nz < 1 || g->ng < 1 || g->nu < 1 || g->nv < 1 || g->nx < 1 || g->n_scatter < 0 ||
      g->n_beams < 1 || g->n_beams > 65535 || !(g->dy > 0) || !(g->dz > 0) || !(g->dx > 0) || !(g->u_max > 0) || !(g->v_max > 0))
    return PBS_ERR_ARG;
  if (precision < PBS_FP64 || precision > PBS_MIXED) return PBS_ERR_ARG;
  for (int f = 0; f < g->ng; f++)
    if (!(g->e_faces[f + 1] > g->e_faces[f])) return PBS_ERR_ARG;
  if (!angular_supported(g->nu, g->nv) || g->nz > 1024 || g->ng > 2048) return PBS_ERR_UNSUPPORTED;
  pbs_ctx *c = new (std::nothrow) pbs_ctx();
  if (!c) return PBS_ERR_NOMEM;
  if (cudaGetDevice(&c->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
    delete c;
    return PBS_ERR_CUDA;
  }
  if (angular_init_tables() != cudaSuccess) {
    delete c;
    return PBS_ERR_CUDA;
  }
  c->stream = (cudaStream_t)stream;
  c->precision = precision;
  c->ny = g->ny; c->nz = g->nz; c->ng = g->ng; c->nu = g->nu; c->nv = g->nv; c->na = g->nu * g->nv;
  c->nx = g->nx; c->K = g->n_scatter;
  c->B = g->n_beams;
  c->beam_steps.assign(c->B, g->nx);
  c->dy = g->dy; c->dz = g->dz; c->dx = g->dx; c->u_max = g->u_max; c->v_max = g->v_max;
  c->du = 2.0 * g->u_max / (g->nu + 1);
  c->dv = 2.0 * g->v_max / (g->nv + 1);
  c->e_faces.assign(g->e_faces, g->e_faces + g->ng + 1);
  c->e_c.resize(g->ng);
  c->de.resize(g->ng);
  for (int k = 0; k < g->ng; k++) {
    c->de[k] = c->e_faces[k + 1] - c->e_faces[k];
    c->e_c[k] = 0.5 * (c->e_faces[k + 1] + c->e_faces[k]);
  }
  c->u.resize(g->nu);
  c->v.resize(g->nv);
  for (int i = 0; i < g->nu; i++) c->u[i] = (i - 0.5 * (g->nu - 1)) * c->du;
  for (int j = 0; j < g->nv; j++) c->v[j] = (j - 0.5 * (g->nv - 1)) * c->dv;
  Dims &d = c->d;
  d.ny = c->ny; d.nz = c->nz; d.ng = c->ng; d.nu = c->nu; d.nv = c->nv; d.na = c->na;
  d.nyz = c->ny * c->nz; d.nbeam = c->B; d.ncomp = c->B * (c->K + 1);
  d.lanes = (long long)d.na * d.nyz;
  d.comp_elems = (long long)d.ng * 2 * d.lanes;
  c->rsize = precision == PBS_FP64 ? 8 : 4;
  c->ssize = precision == PBS_FP64 ? 8 : (precision == PBS_FP32 ? 4 : 2);
  layout(c);
  *out = c;
  return PBS_OK;
}

pbs_status pbs_workspace_size(const pbs_ctx *c, size_t *bytes) {
  if (!c || !bytes) return PBS_ERR_ARG;
  *bytes = c->total;
  return PBS_OK;
}

pbs_status pbs_bind_workspace(pbs_ctx *c, void *p, size_t bytes) {
  if (!c || !p) return fail(c, PBS_ERR_ARG, "null workspace");
  if (bytes < c->total) return fail(c, PBS_ERR_ARG, "workspace too small");
  if (((uintptr_t)p) & 255) return fail(c, PBS_ERR_ARG, "workspace not 256-byte aligned");
  drop_graph(c);
  c->ws = (unsigned char *)p;
  c->ws_bytes = bytes;
  c->have_beam = false;
  c->have_material = false;
  c->pending = false;
  // start from a defined state: zero state, tallies and the device status word
  PBS_CUDA(c, cudaMemsetAsync(c->ws, 0, c->total, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->have_tables) {
    pbs_status r = PBS_DISPATCH(c, upload_tables, c);
    if (r != PBS_OK) return r;
  }
  return PBS_OK;
}

pbs_status pbs_set_physics(pbs_ctx *c, const pbs_physics *ph) {
  if (!c || !ph) return fail(c, PBS_ERR_ARG, "null physics");
  if (!(ph->mp > 0) || !(ph->lambda_p1 > 0) || !(ph->g_beta > 0) || !(ph->g_alpha > 0) || ph->sigma_ct < 0 ||
      ph->s_scale < 0 || ph->ts_scale < 0 || ph->model < 0 || ph->model > 1 || !(ph->t_scale >= 0) ||
      !std::isfinite(ph->t_scale) ||
      (ph->model == 0 && (!(ph->bk_alpha > 0) || !(ph->bk_p > 0) || !(ph->x0 > 0))))
    return fail(c, PBS_ERR_ARG, "physics parameters out of range");
  { pbs_status fr = c->ws ? PBS_DISPATCH(c, flush_impl, c) : PBS_OK; if (fr != PBS_OK) return fr; }
  build_tables(c, *ph);
  c->strag_bound = strag_row_bound(c);
  c->have_tables = true;
  drop_graph(c);
  if (!c->ws) return PBS_OK;  // uploaded at bind time
  return PBS_DISPATCH(c, upload_tables, c);
}

pbs_status pbs_set_tables(pbs_ctx *c, const double *s_face, const double *ts, const double *sig_ct, double lambda_p1,
                          const double *p2) {
  if (!c || !s_face || !ts || !sig_ct) return fail(c, PBS_ERR_ARG, "null table");
  const int G = c->ng;
  if (!(lambda_p1 > 0) || !std::isfinite(lambda_p1)) return fail(c, PBS_ERR_ARG, "lambda_p1 must be > 0");
  for (int f = 0; f <= G; f++)
    if (!(s_face[f] > 0) || !std::isfinite(s_face[f])) return fail(c, PBS_ERR_ARG, "s_face must be finite and > 0");
  for (int g = 0; g < G; g++)
    if (!(ts[g] >= 0) || !(sig_ct[g] >= 0) || !std::isfinite(ts[g]) || !std::isfinite(sig_ct[g]))
      return fail(c, PBS_ERR_ARG, "ts and sig_ct must be finite and >= 0");
  const size_t np2 = (size_t)G * c->na * c->na;
  if (p2) {
    for (size_t e = 0; e < np2; e++)
      if (!std::isfinite(p2[e])) return fail(c, PBS_ERR_ARG, "p2 must be finite");
  } else if (c->K > 0 && c->p2.size() != np2) {
    return fail(c, PBS_ERR_STATE, "no previous P^2: pass p2");
  }
  { pbs_status fr = c->ws ? PBS_DISPATCH(c, flush_impl, c) : PBS_OK; if (fr != PBS_OK) return fr; }
  c->s_base.assign(s_face, s_face + G + 1);
  c->t_face.assign(G + 1, 0.0);  // caller tables replace the built-in straggling too
  fold_straggling(c);
  c->strag_bound = 0.0;
  c->ts.assign(ts, ts + G);
  c->sig.assign(sig_ct, sig_ct + G);
  if (p2) c->p2.assign(p2, p2 + np2);
  transfer_tables(c, lambda_p1);
  c->have_tables = true;
  drop_graph(c);
  if (!c->ws) return PBS_OK;  // uploaded at bind time
  return PBS_DISPATCH(c, upload_tables, c);
}

pbs_status pbs_get_tables(const pbs_ctx *c, double *s_face, double *ts, double *sig, double *p1, double *p2, double *u,
                          double *v) {
  if (!c) return PBS_ERR_ARG;
  if (!c->have_tables) return PBS_ERR_STATE;
  if (s_face) std::memcpy(s_face, c->s_face.data(), 8 * c->s_face.size());
  if (ts) std::memcpy(ts, c->ts.data(), 8 * c->ts.size());
  if (sig) std::memcpy(sig, c->sig.data(), 8 * c->sig.size());
  if (p1) std::memcpy(p1, c->p1.data(), 8 * c->p1.size());
  if (p2) std::memcpy(p2, c->p2.data(), 8 * c->p2.size());
  if (u) std::memcpy(u, c->u.data(), 8 * c->u.size());
  if (v) std::memcpy(v, c->v.data(), 8 * c->v.size());
  return PBS_OK;
}

pbs_status pbs_set_straggling(pbs_ctx *c, const double *t_face) {
  if (!c) return PBS_ERR_ARG;
  if (!c->have_tables) return fail(c, PBS_ERR_STATE, "set the physics or the tables first");
  const int G = c->ng;
  if (t_face)
    for (int f = 0; f <= G; f++)
      if (!(t_face[f] >= 0) || !std::isfinite(t_face[f])) return fail(c, PBS_ERR_ARG, "t_face must be finite and >= 0");
  { pbs_status fr = c->ws ? PBS_DISPATCH(c, flush_impl, c) : PBS_OK; if (fr != PBS_OK) return fr; }
  if (t_face) c->t_face.assign(t_face, t_face + G + 1);
  else c->t_face.assign(G + 1, 0.0);
  fold_straggling(c);
  c->strag_bound = strag_row_bound(c);
  drop_graph(c);
  if (!c->ws) return PBS_OK;
  return PBS_DISPATCH(c, upload_tables, c);
}

pbs_status pbs_get_straggling(const pbs_ctx *c, double *t_face, double *s_base) {
  if (!c) return PBS_ERR_ARG;
  if (!c->have_tables) return PBS_ERR_STATE;
  if (t_face) std::memcpy(t_face, c->t_face.data(), 8 * c->t_face.size());
  if (s_base) std::memcpy(s_base, c->s_base.data(), 8 * c->s_base.size());
  return PBS_OK;
}

pbs_status pbs_set_material(pbs_ctx *c, const double *rho, int n) {
  if (!c || !rho || n < 1 || n > c->nx) return fail(c, PBS_ERR_ARG, "bad material");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "bind a workspace first");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  for (size_t e = 0; e < (size_t)n * c->ny * c->nz; e++)
    if (!(rho[e] >= 0.0) || !std::isfinite(rho[e])) return fail(c, PBS_ERR_ARG, "density must be finite and >= 0");
  pbs_status r = PBS_DISPATCH_R(c, set_material_impl, c, rho, n);
  if (r != PBS_OK) return r;
  c->rho_max = 0.0;
  for (size_t e = 0; e < (size_t)n * c->ny * c->nz; e++) c->rho_max = std::max(c->rho_max, rho[e]);
  c->material_hash = fnv1a(14695981039346656037ULL, rho, (size_t)n * c->ny * c->nz * sizeof(double));
  c->n_slabs = n;
  c->have_material = true;
  return PBS_OK;
}

pbs_status pbs_launch_beam(pbs_ctx *c, const pbs_beam *b) {
  if (!c || !b) return fail(c, PBS_ERR_ARG, "null beam");
  if (!c->ws || !c->have_tables) return fail(c, PBS_ERR_STATE, "bind a workspace and set the physics first");
  std::vector<pbs_beam> all(c->B, *b);
  return pbs_launch_beams(c, all.data(), c->B);
}

pbs_status pbs_launch_beams(pbs_ctx *c, const pbs_beam *beams, int n) {
  if (!c || !beams) return fail(c, PBS_ERR_ARG, "null beams");
  if (n != c->B) return fail(c, PBS_ERR_ARG, "n must equal the context's n_beams");
  if (!c->ws || !c->have_tables) return fail(c, PBS_ERR_STATE, "bind a workspace and set the physics first");
  for (int i = 0; i < n; i++) {
    const pbs_beam *b = beams + i;
    if (!(b->sigma_e > 0) || !(b->sigma_y > 0) || !(b->sigma_z > 0) || !(b->sigma_u > 0) || !(b->sigma_v > 0))
      return fail(c, PBS_ERR_ARG, "beam widths must be > 0");
  }
  pbs_status r = PBS_DISPATCH(c, launch_impl, c, beams);
  if (r != PBS_OK) return r;
  c->have_beam = true;
  return PBS_OK;
}

pbs_status pbs_set_beam_steps(pbs_ctx *c, const int *steps, int n) {
  if (!c || !steps) return fail(c, PBS_ERR_ARG, "null steps");
  if (n != c->B) return fail(c, PBS_ERR_ARG, "n must equal the context's n_beams");
  for (int i = 0; i < n; i++) {
    if (steps[i] < 0 || steps[i] > c->nx) return fail(c, PBS_ERR_ARG, "beam steps must lie in [0, nx]");
    if (i > 0 && steps[i] > steps[i - 1]) return fail(c, PBS_ERR_ARG, "beam steps must be non-increasing");
  }
  if (c->steps_done != 0 || c->pending) return fail(c, PBS_ERR_STATE, "set beam depths before marching");
  c->beam_steps.assign(steps, steps + n);
  drop_graph(c);
  return PBS_OK;
}

pbs_status pbs_run(pbs_ctx *c, int use_graph) {
  if (!c) return PBS_ERR_ARG;
  if (!ready_to_march(c)) return fail(c, PBS_ERR_STATE, "launch a beam (with workspace, physics, material) first");
  if (c->stage != 0) return fail(c, PBS_ERR_STATE, "a staged step is in progress (pbs_step_stage)");
  { pbs_status gr = strag_guard(c, 0.5 * c->dx); if (gr != PBS_OK) return gr; }
  if (use_graph) return PBS_DISPATCH(c, run_graph_impl, c);
  return PBS_DISPATCH(c, run_impl, c);
}

pbs_status pbs_autotune(pbs_ctx *c, int reps) {
  if (!c || reps < 1) return fail(c, PBS_ERR_ARG, "reps must be >= 1");
  if (!ready_to_march(c)) return fail(c, PBS_ERR_STATE, "launch a beam (with workspace, physics, material) first");
  { pbs_status gr = strag_guard(c, 0.5 * c->dx); if (gr != PBS_OK) return gr; }
  return PBS_DISPATCH(c, autotune_impl, c, reps);
}

pbs_status pbs_set_tuning(pbs_ctx *c, const pbs_tuning *t) {
  if (!c || !t) return fail(c, PBS_ERR_ARG, "null tuning");
  if ((t->energy_angles != 4 && t->energy_angles != 8 && t->energy_angles != 16) || t->energy_form < 0 ||
      t->energy_form > 1 || t->transport_ctas < 0 || t->transport_ctas > 64 ||
      (t->transport_cols != 0 && t->transport_cols != 4 && t->transport_cols != 6 && t->transport_cols != 8) ||
      t->angular_form < 0 ||
      t->angular_form > 7 || t->source_form < 0 || t->source_form > 2)
    return fail(c, PBS_ERR_ARG, "tuning value out of range");
  c->tune = *t;
  drop_graph(c);
  return PBS_OK;
}

pbs_status pbs_set_options(pbs_ctx *c, const pbs_options *o) {
  if (!c || !o) return fail(c, PBS_ERR_ARG, "null options");
  if (o->angular_integrator < 0 || o->angular_integrator > 1) return fail(c, PBS_ERR_ARG, "unknown angular integrator");
  if (o->transport_integrator < 0 || o->transport_integrator > 1)
    return fail(c, PBS_ERR_ARG, "unknown transport integrator");
  if (o->straggling_integrator < 0 || o->straggling_integrator > 1)
    return fail(c, PBS_ERR_ARG, "unknown straggling integrator");
  if (o->transport_integrator == 1 && c->nz > 256)
    return fail(c, PBS_ERR_UNSUPPORTED, "the Crank-Nicolson transport sweep takes rows of at most 256 columns");
  { pbs_status fr = c->ws ? PBS_DISPATCH(c, flush_impl, c) : PBS_OK; if (fr != PBS_OK) return fr; }
  c->opts = *o;
  drop_graph(c);
  return PBS_OK;
}

pbs_status pbs_get_options(const pbs_ctx *c, pbs_options *o) {
  if (!c || !o) return PBS_ERR_ARG;
  *o = c->opts;
  return PBS_OK;
}

pbs_status pbs_get_tuning(const pbs_ctx *c, pbs_tuning *t) {
  if (!c || !t) return PBS_ERR_ARG;
  *t = c->tune;
  return PBS_OK;
}

pbs_status pbs_step(pbs_ctx *c, int n) {
  if (!c || n < 0) return fail(c, PBS_ERR_ARG, "bad step count");
  if (!ready_to_march(c)) return fail(c, PBS_ERR_STATE, "launch a beam (with workspace, physics, material) first");
  if (c->stage != 0) return fail(c, PBS_ERR_STATE, "a staged step is in progress (pbs_step_stage)");
  if (c->steps_done + n > c->n_slabs) return fail(c, PBS_ERR_ARG, "march would pass the last material slab");
  { pbs_status gr = strag_guard(c, 0.5 * c->dx); if (gr != PBS_OK) return gr; }
  return PBS_DISPATCH(c, step_impl, c, n);
}

pbs_status pbs_step_stage(pbs_ctx *c, int stage) {
  if (!c || stage < 0 || stage > 3) return fail(c, PBS_ERR_ARG, "stage must be 0..3");
  if (!ready_to_march(c)) return fail(c, PBS_ERR_STATE, "launch a beam (with workspace, physics, material) first");
  if (stage != c->stage) return fail(c, PBS_ERR_STATE, "stages of a step run in order 0, 1, 2, 3");
  if (stage == 0) {
    if (c->steps_done + 1 > c->n_slabs) return fail(c, PBS_ERR_ARG, "march would pass the last material slab");
    pbs_status gr = strag_guard(c, 0.5 * c->dx);
    if (gr != PBS_OK) return gr;
  }
  pbs_status r = PBS_DISPATCH(c, stage_impl, c, stage);
  if (r == PBS_OK) c->stage = (stage + 1) & 3;
  return r;
}

pbs_status pbs_set_lateral_part(pbs_ctx *c, int y_offset, int ny_global, int halo_lo, int halo_hi) {
  if (!c) return PBS_ERR_ARG;
  if (c->B != 1) return fail(c, PBS_ERR_UNSUPPORTED, "a lateral part holds one beam (n_beams = 1)");
  if (ny_global < c->ny || y_offset < 0 || y_offset + c->ny > ny_global || halo_lo < 0 || halo_hi < 0 ||
      halo_lo + halo_hi >= c->ny || (y_offset == 0) != (halo_lo == 0) ||
      (y_offset + c->ny == ny_global) != (halo_hi == 0))
    return fail(c, PBS_ERR_ARG,
                "bad lateral part: rows must lie inside the grid, with halo rows exactly on the interior sides");
  if (c->have_beam) return fail(c, PBS_ERR_STATE, "declare the lateral part before launching the beam");
  c->part = !(y_offset == 0 && ny_global == c->ny);
  c->part_y0 = y_offset;
  c->part_nyg = ny_global;
  c->halo_lo = halo_lo;
  c->halo_hi = halo_hi;
  return PBS_OK;
}

pbs_status pbs_copy_rows(pbs_ctx *c, int first_row, int n_rows, int to_buffer, void *dev_buf) {
  if (!c || !dev_buf || first_row < 0 || n_rows < 0 || first_row + n_rows > c->ny)
    return fail(c, PBS_ERR_ARG, "rows out of range or null buffer");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  if (n_rows == 0) return PBS_OK;
  const size_t row = (size_t)c->nz * c->rsize, pitch = (size_t)c->ny * row;
  const size_t planes = (size_t)c->d.ncomp * c->ng * 2 * c->na;
  unsigned char *w = at<unsigned char>(c, c->off_psi) + (size_t)first_row * row;
  unsigned char *b = static_cast<unsigned char *>(dev_buf);
  const size_t width = (size_t)n_rows * row;
  for (size_t p0 = 0; p0 < planes; p0 += 32768) {
    const size_t np = std::min<size_t>(32768, planes - p0);
    if (to_buffer)
      PBS_CUDA(c, cudaMemcpy2DAsync(b + p0 * width, width, w + p0 * pitch, pitch, width, np, cudaMemcpyDefault,
                                    c->stream));
    else
      PBS_CUDA(c, cudaMemcpy2DAsync(w + p0 * pitch, pitch, b + p0 * width, width, width, np, cudaMemcpyDefault,
                                    c->stream));
  }
  return PBS_OK;
}

pbs_status pbs_domain_step(pbs_ctx *const *parts, int n_parts, int n_steps) {
  if (!parts || n_parts < 1 || n_steps < 0) return PBS_ERR_ARG;
  for (int i = 0; i < n_parts; i++)
    if (!parts[i]) return PBS_ERR_ARG;
  pbs_ctx *c0 = parts[0];
  const int nyg = c0->part ? c0->part_nyg : c0->ny;
  int owned_end = 0;
  for (int i = 0; i < n_parts; i++) {
    pbs_ctx *c = parts[i];
    if (!ready_to_march(c)) return fail(c0, PBS_ERR_STATE, "every part needs a launched beam, material and tables");
    if (c->stage != 0) return fail(c0, PBS_ERR_STATE, "a staged step is in progress on a part");
    if (c->B != 1 || c->precision != c0->precision || c->nz != c0->nz || c->ng != c0->ng || c->na != c0->na ||
        c->K != c0->K || c->dx != c0->dx || c->dy != c0->dy || c->dz != c0->dz || c->u_max != c0->u_max ||
        c->v_max != c0->v_max)
      return fail(c0, PBS_ERR_ARG, "parts differ in grid, precision or scattering order");
    if (std::memcmp(&c->opts, &c0->opts, sizeof(pbs_options)) != 0)
      return fail(c0, PBS_ERR_ARG, "parts differ in method options");
    if (c->opts.transport_integrator != 0)
      return fail(c0, PBS_ERR_UNSUPPORTED,
                  "the Crank-Nicolson transport sweeps whole rows: no finite halo; use the explicit trapezoid");
    if (c->steps_done != c0->steps_done || c->pending != c0->pending || beam_depth(c, 0) != beam_depth(c0, 0))
      return fail(c0, PBS_ERR_STATE, "parts are at different depths");
    if (n_parts > 1 && (!c->part || c->part_nyg != nyg))
      return fail(c0, PBS_ERR_ARG, "declare every part with pbs_set_lateral_part on one grid");
    // owned rows tile the grid in order; interior halos cover the transport's reach
    const int y0 = n_parts > 1 ? c->part_y0 : 0;
    if (y0 + c->halo_lo != owned_end) return fail(c0, PBS_ERR_ARG, "parts must follow one another in y");
    owned_end = y0 + c->ny - c->halo_hi;
    const int owned = c->ny - c->halo_lo - c->halo_hi;
    if ((i > 0 && c->halo_lo < kHaloRows) || (i + 1 < n_parts && c->halo_hi < kHaloRows))
      return fail(c0, PBS_ERR_ARG, "interior halos need at least 4 rows (the reach of the two transport stages)");
    if ((i > 0 && parts[i - 1]->halo_hi > owned) || (i + 1 < n_parts && parts[i + 1]->halo_lo > owned))
      return fail(c0, PBS_ERR_ARG, "a neighbour's halo is wider than this part's own rows");
    if (c->steps_done + n_steps > c->n_slabs) return fail(c0, PBS_ERR_ARG, "march would pass the last material slab");
    pbs_status gr = strag_guard(c, 0.5 * c->dx);
    if (gr != PBS_OK) return gr;
  }
  if (owned_end != nyg) return fail(c0, PBS_ERR_ARG, "the parts do not cover the grid");
  return PBS_DISPATCH(c0, domain_step_impl, parts, n_parts, n_steps);
}

pbs_status pbs_batch_workspace_size(pbs_ctx *const *beams, int n_beams, size_t *bytes) {
  if (!beams || n_beams < 1 || !bytes) return PBS_ERR_ARG;
  for (int i = 0; i < n_beams; i++)
    if (!beams[i]) return PBS_ERR_ARG;
  // the larger of the two layouts (pipelined passes have more tasks and counters)
  *bytes = std::max(batch_layout(beams, n_beams, 0).total, batch_layout(beams, n_beams, 1).total);
  return PBS_OK;
}

pbs_status pbs_run_batch(pbs_ctx *const *beams, int n_beams, void *dev_ws, size_t bytes, const pbs_batch_options *o) {
  if (!beams || n_beams < 1 || n_beams > 65535) return PBS_ERR_ARG;
  for (int i = 0; i < n_beams; i++)
    if (!beams[i]) return PBS_ERR_ARG;
  const pbs_batch_options def{0, 0.0, -1, 0, 0, 0};
  return run_batch_impl(beams, n_beams, dev_ws, bytes, o ? *o : def, -1);
}

pbs_status pbs_batch_autotune(pbs_ctx *const *beams, int n_beams, void *dev_ws, size_t bytes, int steps,
                              pbs_batch_options *opts) {
  if (!beams || n_beams < 1 || n_beams > 65535 || !opts || steps < 1) return PBS_ERR_ARG;
  for (int i = 0; i < n_beams; i++)
    if (!beams[i]) return PBS_ERR_ARG;
  pbs_ctx *c0 = beams[0];
  // the candidates: shape 0 (4 columns), shape 1 with 4 and, where some row
  // splits into 6-column lanes, with 6 columns
  bool six = false;
  for (int i = 0; i < n_beams; i++) six = six || beams[i]->nz % 6 == 0;
  const int cand[6][3] = {{0, 4, 0}, {1, 4, 0}, {1, 6, 0}, {0, 4, 1}, {1, 4, 1}, {1, 6, 1}};
  bool big = false;  // 16 x 16 angles: shape 0 only
  for (int i = 0; i < n_beams; i++) big = big || std::max(beams[i]->nu, beams[i]->nv) > 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PBS_CUDA(c0, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c0, PBS_ERR_CUDA, "event create");
  }
  const bool prof = c0->profiling;
  c0->profiling = false;
  pbs_status r = PBS_OK;
  float best = 1e30f;
  pbs_batch_options pick = *opts, trial = *opts;
  trial.use_graph = 0;
  trial.hold_beam = -1;
  for (int k = 0; k < 6 && r == PBS_OK; k++) {
    if (cand[k][1] == 6 && !six) continue;
    if (big && cand[k][0] != 0) continue;
    trial.shape = cand[k][0];
    trial.transport_cols = cand[k][1];
    trial.pipeline = cand[k][2];
    for (int rep = 0; rep < 2 && r == PBS_OK; rep++) {
      cudaEventRecord(e0, c0->stream);
      r = run_batch_impl(beams, n_beams, dev_ws, bytes, trial, steps);
      cudaEventRecord(e1, c0->stream);
      if (r != PBS_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) { r = fail(c0, PBS_ERR_CUDA, "batch trial"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        pick.shape = trial.shape;
        pick.transport_cols = trial.transport_cols;
        pick.pipeline = trial.pipeline;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c0->profiling = prof;
  if (r != PBS_OK) return r;
  // the trials marched the beams: restart them from their projections
  for (int b = 0; b < n_beams; b++) {
    pbs_status q = beams[b]->precision == PBS_FP32 ? reinit_impl<float, float>(beams[b])
                                                   : reinit_impl<float, __nv_bfloat16>(beams[b]);
    if (q != PBS_OK) return q;
  }
  PBS_CUDA(c0, cudaStreamSynchronize(c0->stream));
  for (int b = 0; b < n_beams; b++) {
    pbs_status q = check_device_status(beams[b]);
    if (q != PBS_OK) return q;
  }
  opts->shape = pick.shape;
  opts->transport_cols = pick.transport_cols;
  opts->pipeline = pick.pipeline;
  return PBS_OK;
}

pbs_status pbs_flush(pbs_ctx *c) {
  if (!c) return PBS_ERR_ARG;
  if (!c->ws) return PBS_OK;
  return PBS_DISPATCH(c, flush_impl, c);
}

pbs_status pbs_checkpoint_size(const pbs_ctx *c, size_t *bytes) {
  if (!c || !bytes) return PBS_ERR_ARG;
  *bytes = ckpt_bytes(c);
  return PBS_OK;
}

pbs_status pbs_checkpoint_save(pbs_ctx *c, void *host, size_t bytes) {
  if (!c || !host) return fail(c, PBS_ERR_ARG, "null buffer");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  if (bytes < ckpt_bytes(c)) return fail(c, PBS_ERR_ARG, "buffer smaller than pbs_checkpoint_size");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "PBSCKPT1", 8);
  h.version = 2;
  h.precision = c->precision;
  h.ny = c->ny; h.nz = c->nz; h.ng = c->ng; h.nu = c->nu; h.nv = c->nv; h.nx = c->nx; h.K = c->K; h.B = c->B;
  h.steps_done = c->steps_done;
  h.pending = c->pending ? 1 : 0;
  h.have_beam = c->have_beam ? 1 : 0;
  h.n_slabs_at_save = c->n_slabs;
  h.angular_integrator = c->opts.angular_integrator;
  h.transport_integrator = c->opts.transport_integrator;
  h.straggling_integrator = c->opts.straggling_integrator;
  h.tables_hash = c->have_tables ? tables_hash(c) : 0;
  h.material_hash = c->have_material ? c->material_hash : 0;
  unsigned char *p = static_cast<unsigned char *>(host);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t nyz = (size_t)c->ny * c->nz;
  const size_t parts[4][2] = {{c->off_psi, (size_t)c->d.ncomp * c->d.comp_elems * c->rsize},
                              {c->off_dose, (size_t)c->B * c->nx * nyz * 8},
                              {c->off_flu, (size_t)c->B * (c->nx + 1) * nyz * 8},
                              {c->off_init, (size_t)c->B * init_stride(c) * 8}};
  for (auto &q : parts) {
    PBS_CUDA(c, cudaMemcpyAsync(p, at<void>(c, q[0]), q[1], cudaMemcpyDeviceToHost, c->stream));
    p += q[1];
  }
  std::memcpy(p, c->beam_steps.data(), (size_t)c->B * sizeof(int));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_status(c);
}

pbs_status pbs_checkpoint_load(pbs_ctx *c, const void *host, size_t bytes) {
  if (!c || !host) return fail(c, PBS_ERR_ARG, "null buffer");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  if (bytes < sizeof(CkptHeader)) return fail(c, PBS_ERR_ARG, "not a checkpoint");
  CkptHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "PBSCKPT1", 8) != 0 || h.version != 2) return fail(c, PBS_ERR_ARG, "not a checkpoint");
  if (h.precision != c->precision || h.ny != c->ny || h.nz != c->nz || h.ng != c->ng || h.nu != c->nu ||
      h.nv != c->nv || h.nx != c->nx || h.K != c->K || h.B != c->B)
    return fail(c, PBS_ERR_ARG, "checkpoint of another grid, precision or batch");
  if (bytes < ckpt_bytes(c)) return fail(c, PBS_ERR_ARG, "truncated checkpoint");
  const int *steps = reinterpret_cast<const int *>(static_cast<const unsigned char *>(host) + ckpt_bytes(c) -
                                                   (size_t)c->B * sizeof(int));
  for (int b = 0; b < c->B; b++)
    if (steps[b] < 0 || steps[b] > c->nx || (b > 0 && steps[b] > steps[b - 1]))
      return fail(c, PBS_ERR_ARG, "corrupt checkpoint (beam depths)");
  if (h.steps_done < 0 || h.steps_done > c->nx) return fail(c, PBS_ERR_ARG, "corrupt checkpoint (depth)");
  if ((h.pending != 0 && h.pending != 1) || (h.have_beam != 0 && h.have_beam != 1))
    return fail(c, PBS_ERR_ARG, "corrupt checkpoint (flags)");
  // a deferred closing half belongs to step steps_done - 1 of a beam that marched it
  if (h.pending && (h.steps_done < 1 || h.steps_done > steps[0] || !h.have_beam))
    return fail(c, PBS_ERR_ARG, "corrupt checkpoint (deferred half without a marched step)");
  if (!c->have_tables || !c->have_material)
    return fail(c, PBS_ERR_STATE, "set the tables and the material before restoring a checkpoint");
  if (h.angular_integrator != c->opts.angular_integrator || h.transport_integrator != c->opts.transport_integrator ||
      h.straggling_integrator != c->opts.straggling_integrator)
    return fail(c, PBS_ERR_ARG, "checkpoint marched with other method options (pbs_set_options)");
  if (h.tables_hash != tables_hash(c)) return fail(c, PBS_ERR_ARG, "checkpoint marched with other tables");
  if (h.material_hash != c->material_hash || h.n_slabs_at_save != c->n_slabs)
    return fail(c, PBS_ERR_ARG, "checkpoint marched through another density field");
  const unsigned char *p = static_cast<const unsigned char *>(host) + sizeof(h);
  const size_t nyz = (size_t)c->ny * c->nz;
  const size_t parts[4][2] = {{c->off_psi, (size_t)c->d.ncomp * c->d.comp_elems * c->rsize},
                              {c->off_dose, (size_t)c->B * c->nx * nyz * 8},
                              {c->off_flu, (size_t)c->B * (c->nx + 1) * nyz * 8},
                              {c->off_init, (size_t)c->B * init_stride(c) * 8}};
  for (auto &q : parts) {
    PBS_CUDA(c, cudaMemcpyAsync(at<void>(c, q[0]), p, q[1], cudaMemcpyHostToDevice, c->stream));
    p += q[1];
  }
  PBS_CUDA(c, cudaMemsetAsync(at<void>(c, c->off_err), 0, 64, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  c->beam_steps.assign(steps, steps + c->B);
  c->steps_done = h.steps_done;
  c->pending = h.pending != 0;
  c->have_beam = h.have_beam != 0;
  drop_graph(c);
  return PBS_OK;
}

pbs_status pbs_get_depth(const pbs_ctx *c, int *s) {
  if (!c || !s) return PBS_ERR_ARG;
  *s = c->steps_done;
  return PBS_OK;
}

pbs_status pbs_read_dose(pbs_ctx *c, double *out, size_t n) {
  if (!c || !out) return fail(c, PBS_ERR_ARG, "null output");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  const size_t per = (size_t)c->B * c->ny * c->nz;
  if (n == 0 || n % per != 0 || n / per > (size_t)c->nx) return fail(c, PBS_ERR_ARG, "n must be n_beams*n_slabs*ny*nz");
  const size_t row = n / c->B * 8;  // bytes of one beam's slabs
  PBS_CUDA(c, cudaMemcpy2DAsync(out, row, at<void>(c, c->off_dose), (size_t)c->nx * c->ny * c->nz * 8, row, c->B,
                                cudaMemcpyDeviceToHost, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_status(c);
}

pbs_status pbs_read_fluence(pbs_ctx *c, double *out, size_t n) {
  if (!c || !out) return fail(c, PBS_ERR_ARG, "null output");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  const size_t per = (size_t)c->B * c->ny * c->nz;
  if (n == 0 || n % per != 0 || n / per > (size_t)c->steps_done + 1)
    return fail(c, PBS_ERR_ARG, "n must be n_beams*n_planes*ny*nz");
  const size_t row = n / c->B * 8;
  PBS_CUDA(c, cudaMemcpy2DAsync(out, row, at<void>(c, c->off_flu), (size_t)(c->nx + 1) * c->ny * c->nz * 8, row, c->B,
                                cudaMemcpyDeviceToHost, c->stream));
  PBS_CUDA(c, cudaStreamSynchronize(c->stream));
  return check_device_status(c);
}

pbs_status pbs_read_psi(pbs_ctx *c, int k, double *out, size_t n) {
  if (!c || !out || k < 0 || k >= c->d.ncomp) return fail(c, PBS_ERR_ARG, "bad component");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  if (n != (size_t)c->d.comp_elems) return fail(c, PBS_ERR_ARG, "n must be ng*2*nu*nv*ny*nz");
  return PBS_DISPATCH_R(c, read_psi_impl, c, k, out);
}

pbs_status pbs_write_psi(pbs_ctx *c, int k, const double *in, size_t n) {
  if (!c || !in || k < 0 || k >= c->d.ncomp) return fail(c, PBS_ERR_ARG, "bad component");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "no workspace");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  if (n != (size_t)c->d.comp_elems) return fail(c, PBS_ERR_ARG, "n must be ng*2*nu*nv*ny*nz");
  return PBS_DISPATCH_R(c, write_psi_impl, c, k, in);
}

pbs_status pbs_substep_energy(pbs_ctx *c, double h, int slab, int flu_plane) {
  if (!c || !(h >= 0) || slab < 0 || slab >= c->n_slabs || flu_plane > c->nx)
    return fail(c, PBS_ERR_ARG, "bad substep arguments");
  if (!c->ws || !c->have_tables || !c->have_material) return fail(c, PBS_ERR_STATE, "not set up");
  { pbs_status gr = strag_guard(c, h); if (gr != PBS_OK) return gr; }
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  return PBS_DISPATCH(c, energy_all, c, h, slab, flu_plane);
}

pbs_status pbs_substep_transport(pbs_ctx *c, double h) {
  if (!c || !(h >= 0)) return fail(c, PBS_ERR_ARG, "bad substep arguments");
  if (!c->ws) return fail(c, PBS_ERR_STATE, "not set up");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  return PBS_DISPATCH_R(c, transport_all, c, h);
}

pbs_status pbs_substep_angular(pbs_ctx *c, double h, int slab) {
  if (!c || !(h >= 0) || slab < 0 || slab >= c->n_slabs) return fail(c, PBS_ERR_ARG, "bad substep arguments");
  if (!c->ws || !c->have_tables || !c->have_material) return fail(c, PBS_ERR_STATE, "not set up");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  return PBS_DISPATCH_R(c, angular_all, c, h, slab);
}

pbs_status pbs_eval_source(pbs_ctx *c, int k_from, int slab, double *out, size_t n) {
  if (!c || !out || k_from < 0 || k_from >= c->d.ncomp || slab < 0 || slab >= c->n_slabs)
    return fail(c, PBS_ERR_ARG, "bad arguments");
  if (c->K < 1) return fail(c, PBS_ERR_STATE, "the context has no scattered component (n_scatter = 0)");
  if (!c->ws || !c->have_tables || !c->have_material) return fail(c, PBS_ERR_STATE, "not set up");
  { pbs_status fr = PBS_DISPATCH(c, flush_impl, c); if (fr != PBS_OK) return fr; }
  if (n != (size_t)c->ng * c->na * c->ny * c->nz) return fail(c, PBS_ERR_ARG, "n must be ng*nu*nv*ny*nz");
  return PBS_DISPATCH(c, eval_source_impl, c, k_from, slab, out);
}

pbs_status pbs_kernel_launches(const pbs_ctx *c, long long *count) {
  if (!c || !count) return PBS_ERR_ARG;
  *count = c->launches;
  return PBS_OK;
}

pbs_status pbs_set_profiling(pbs_ctx *c, int on) {
  if (!c) return PBS_ERR_ARG;
  pbs_status r = fold_profile(c);
  if (r != PBS_OK) return r;
  c->batch_prof = nullptr;
  c->profiling = on != 0;
  for (int k = 0; k < PBS_KERNEL_KINDS; k++) {
    c->prof_count[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  return PBS_OK;
}

pbs_status pbs_profile_read(pbs_ctx *c, int kind, long long *count, double *total_ms) {
  if (!c || kind < 0 || kind >= PBS_KERNEL_KINDS || !count || !total_ms) return fail(c, PBS_ERR_ARG, "bad kind");
  pbs_status r = fold_profile(c);
  if (r != PBS_OK) return r;
  *count = c->prof_count[kind];
  *total_ms = c->prof_ms[kind];
  return PBS_OK;
}

const char *pbs_last_error(const pbs_ctx *c) { return c ? c->err.c_str() : "null context"; }

const char *pbs_status_string(int s) {
  switch (s) {
    case PBS_OK: return "ok";
    case PBS_ERR_ARG: return "invalid argument";
    case PBS_ERR_CUDA: return "CUDA error";
    case PBS_ERR_NOMEM: return "out of memory";
    case PBS_ERR_STATE: return "call out of order";
    case PBS_ERR_TIMEOUT: return "device wait timed out";
    case PBS_ERR_UNSUPPORTED: return "unsupported grid";
  }
  return "unknown status";
}

void pbs_destroy(pbs_ctx *c) { delete c; }

}  // extern "C"
