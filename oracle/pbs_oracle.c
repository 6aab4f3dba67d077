/*
 * pbs_oracle.c -- plain FP64 CPU oracle of the depth-marching proton-beam
 * solver of Zhang, Bai & Tang, "A deterministic solver for the linear
 * Boltzmann model of a single mono-directional proton beam"
 * (arXiv 2504.00340).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table generator
 * with the CUDA library; both are written separately from the paper.
 *
 * Everything here is double precision, written as straightforward loops in
 * the paper's order and notation.  OpenMP (when compiled with -fopenmp) only
 * runs the independent index sets that Remark 2 names in parallel; each
 * output element is still computed by exactly the same sequence of
 * operations as in a serial run.
 *
 * Readings of the paper that the paper leaves open are marked "Reading:".
 *
 * Data layout of one component psi_k (logical, row-major):
 *     psi[g][c][j][i][p][q]
 *   g = energy group 0..G-1 (0 = lowest energy; the paper's g = G is the top)
 *   c = DG coefficient 0 (psi^1, group mean) or 1 (psi^2, slope)
 *   j,i = angle indices in v and u (u fastest of the two)
 *   p,q = lateral cell indices in y and z (z fastest)
 *
 * Parity status: every function below is pinned by a CPU test against a
 * closed form, an invariant, a special case that reduces to a library
 * routine, or brute force (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "pbs_oracle.h"

#define IDX5(ctx, g, c, a, p, q) \
  (((((size_t)(g) * 2 + (c)) * (size_t)(ctx)->na + (a)) * (size_t)(ctx)->ny + (p)) * (size_t)(ctx)->nz + (q))

struct orc_ctx {
  int ny, nz, ng, nu, nv, na;
  double dy, dz, du, dv, u_max, v_max;
  orc_phys ph;
  double *e_faces;  /* ng+1 */
  double *e_c;      /* group centre E_g */
  double *de;       /* group width Delta E_g */
  double *s_face;   /* mass stopping power at the faces, ng+1, with the straggling drift folded in */
  double *s_base;   /* mass stopping power at the faces, ng+1, as tabulated */
  double *t_face;   /* mass straggling coefficient at the faces, ng+1 (0: no straggling) */
  int strag_on;     /* any t_face != 0 */
  int strag_cn;     /* straggling time integrator: 0 explicit inside CN, 1 Crank-Nicolson */
  double *ts;       /* group-averaged scattering power, ng */
  double *sig;      /* catastrophic removal (mass), ng */
  double *p1;       /* [gp][g] probability of gp -> g */
  double *p2;       /* [g][a][ap] density in (u,v) of ap -> a */
  double *u, *v;    /* angle nodes */
  int angular_exact; /* angular time integrator: 0 Crank-Nicolson, 1 exact exponential */
  int transport_cn;  /* transport time integrator: 0 explicit trapezoid, 1 CN with lagged slope */
};

/* Angular time integrator (Section 3.4: the paper integrates each sine mode
 * with "an ODE solver"; Section 3.3 prescribes Crank-Nicolson): 0 keeps CN,
 * 1 takes each mode's exact solution exp(h kappa lam / 2). */
void orc_set_angular_exact(orc_ctx *c, int exact) { c->angular_exact = exact != 0; }

/* ------------------------------------------------------------------ */
/* Physics tables (Appendix A with the Bragg-Kleeman and Highland      */
/* substitutions of the workloads; Section 4, Appendix A.4)            */
/* ------------------------------------------------------------------ */

/* Mass stopping power from the Bragg-Kleeman range law R(E) = alpha E^p:
 * S = dE / d(rho x) = 1 / (dR/dE) = E^(1-p) / (alpha p). */
static double bk_stopping(const orc_phys *ph, double e) {
  return ph->s_scale * pow(e, 1.0 - ph->bk_p) / (ph->bk_alpha * ph->bk_p);
}

/* Antiderivative in E of the Highland-type scattering power
 *   T_s(E) = (Es / (p v))^2 / X0,  p v = E (E + 2M) / (E + M),
 * written with w = E + M as (Es^2/X0) w^2 / (w^2 - M^2)^2, whose primitive is
 *   (Es^2/X0) [ ln((w-M)/(w+M)) / (4M) - w / (2 (w^2 - M^2)) ]. */
static double highland_primitive(const orc_phys *ph, double e) {
  double m = ph->mp, w = e + m;
  double k = ph->es * ph->es / ph->x0;
  return k * (log((w - m) / (w + m)) / (4.0 * m) - w / (2.0 * (w * w - m * m)));
}

double orc_highland(const orc_phys *ph, double e) {
  double m = ph->mp;
  double pv = e * (e + 2.0 * m) / (e + m);
  return ph->ts_scale * (ph->es / pv) * (ph->es / pv) / ph->x0;
}

/* The paper's own tables (Appendix A), for water as the paper's examples.
 * Stopping power: Bethe-Bloch per element with the density correction taken
 * as 0 (protons of at most a few hundred MeV) and the piecewise I-value rule
 * of Appendix A.1, combined by Bragg additivity over the mass fractions.
 * Scattering: the screened-Rutherford momentum-transfer cross section of
 * Appendix A.3 per atom, summed over the atoms of one gram; with
 * (rho sigma_tr / 2)(d_uu + d_vv) it is the growth of <u^2> per unit
 * density and length, the same role as the Highland power. */
#define ORC_ME 0.51099895   /* electron rest energy, MeV */
#define ORC_KB 0.307075     /* 4 pi N_A r_e^2 m_e c^2, MeV cm^2 / mol */
#define ORC_E2 1.439964e-13 /* e^2 / (4 pi eps0), MeV cm */
#define ORC_FS (1.0 / 137.035999)
#define ORC_NA 6.02214076e23
#define ORC_AMU 931.494     /* MeV per atomic mass unit */

/* Z, A (g/mol), mass fraction of water */
static const double orc_water[2][3] = {{1.0, 1.00794, 0.111894}, {8.0, 15.9994, 0.888106}};

static double i_value_mev(double z) {
  double ev = (z < 1.5) ? 19.0 : (z <= 13.0 ? 11.2 + 11.7 * z : 52.8 + 8.71 * z);
  return ev * 1e-6;
}

double orc_bethe_element(const orc_phys *ph, double z, double a, double e) {
  double gam = 1.0 + e / ph->mp, b2 = 1.0 - 1.0 / (gam * gam);
  return ORC_KB * z / a / b2 * (log(2.0 * ORC_ME * b2 * gam * gam / i_value_mev(z)) - b2);
}

double orc_bethe_water(const orc_phys *ph, double e) {
  double s = 0.0;
  for (int k = 0; k < 2; k++) s += orc_water[k][2] * orc_bethe_element(ph, orc_water[k][0], orc_water[k][1], e);
  return s;
}

double orc_sigma_tr_element(const orc_phys *ph, double z, double a, double e) {
  double gam = 1.0 + e / ph->mp, b2 = 1.0 - 1.0 / (gam * gam);
  double mt = a * ORC_AMU;                 /* target nucleus */
  double m0 = ph->mp * mt / (ph->mp + mt); /* reduced mass */
  double r = z * ORC_E2 / (m0 * b2);       /* z_i Z e^2 / (4 pi eps0 m0 v^2), z_i = 1 */
  double p = sqrt(e * (e + 2.0 * ph->mp)); /* MeV / c */
  double th = cbrt(z) * ORC_FS * ORC_ME / p;
  double eta = th * th;
  return 2.0 * 3.14159265358979323846 * r * r * (log((eta + 1.0) / eta) - 1.0 / (eta + 1.0));
}

double orc_scat_power_water(const orc_phys *ph, double e) {
  double s = 0.0;
  for (int k = 0; k < 2; k++)
    s += ORC_NA * orc_water[k][2] / orc_water[k][1] * orc_sigma_tr_element(ph, orc_water[k][0], orc_water[k][1], e);
  return s;
}

/* Energy-straggling coefficient of Appendix A.2 (Williams' form of Bohr's
 * formula with the binding correction), per gram of water: the per-electron
 *   4 pi e^4 (1 + 4 I / (3 m_e v^2) ln(2 m_e v^2 / I))
 * times the electrons per gram N_A Z / A of each element, with that
 * element's I-value (the piecewise rule of Appendix A.1), summed over the
 * mass fractions.  m_e v^2 = m_e c^2 beta^2.  MeV^2 cm^2 / g. */
double orc_williams_water(const orc_phys *ph, double e) {
  double gam = 1.0 + e / ph->mp, b2 = 1.0 - 1.0 / (gam * gam);
  double mv2 = ORC_ME * b2, s = 0.0;
  for (int k = 0; k < 2; k++) {
    double z = orc_water[k][0], a = orc_water[k][1], w = orc_water[k][2], i = i_value_mev(z);
    s += w * z / a * (1.0 + 4.0 * i / (3.0 * mv2) * log(2.0 * mv2 / i));
  }
  return 4.0 * 3.14159265358979323846 * ORC_E2 * ORC_E2 * ORC_NA * s;
}

/* Section 3.2 splits the straggling term (1/2) d^2(T psi)/dE^2 into
 * (1/2) d/dE(T dpsi/dE), taken by the interior-penalty form below, and
 * (1/2) d/dE(T' psi), which the paper treats like the stopping-power term.
 * Reading: it IS the stopping-power operator with S replaced by T'/2, so
 * the two drifts add at every face: S_eff = S + T'/2.  T is linear in each
 * group through its face values (as S, Eq. appSE), so T' is the group's
 * slope; at an inner face it is the mean of the two neighbouring slopes
 * (on a uniform grid the paper's (T_{g+1} - T_g) / dE of centre values),
 * at the two outer faces the one adjacent slope. */
static void fold_straggling(orc_ctx *c) {
  int G = c->ng;
  c->strag_on = 0;
  for (int f = 0; f <= G; f++) {
    double tp;
    if (G == 1) tp = (c->t_face[1] - c->t_face[0]) / c->de[0];
    else if (f == 0) tp = (c->t_face[1] - c->t_face[0]) / c->de[0];
    else if (f == G) tp = (c->t_face[G] - c->t_face[G - 1]) / c->de[G - 1];
    else tp = 0.5 * ((c->t_face[f] - c->t_face[f - 1]) / c->de[f - 1] + (c->t_face[f + 1] - c->t_face[f]) / c->de[f]);
    c->s_face[f] = c->s_base[f] + 0.5 * tp;
    if (c->t_face[f] != 0.0) c->strag_on = 1;
  }
}

/* Caller-given straggling coefficients at the faces (NULL: none). */
void orc_set_straggling_table(orc_ctx *c, const double *t_face) {
  for (int f = 0; f <= c->ng; f++) c->t_face[f] = t_face ? t_face[f] : 0.0;
  fold_straggling(c);
}

/* Straggling time integrator inside the energy substep: 0 treats the
 * interior-penalty part explicitly (old state only) inside the CN step of
 * the rest of the energy operator, 1 takes it into the CN step as well. */
void orc_set_straggling_cn(orc_ctx *c, int full) { c->strag_cn = full != 0; }

void orc_get_straggling(const orc_ctx *c, double *t_face, double *s_base) {
  if (t_face) memcpy(t_face, c->t_face, sizeof(double) * (c->ng + 1));
  if (s_base) memcpy(s_base, c->s_base, sizeof(double) * (c->ng + 1));
}

/* Gamma density of the catastrophic deflection angle (Appendix A.4). */
static double gamma_pdf(double th, double al, double be) {
  if (th <= 0.0) return (al == 1.0) ? be : 0.0;
  return pow(be, al) / tgamma(al) * pow(th, al - 1.0) * exp(-be * th);
}

orc_ctx *orc_create(const orc_grid *gr, const orc_phys *ph) {
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  int G = gr->ng, na;
  if (!c) return NULL;
  c->ny = gr->ny; c->nz = gr->nz; c->ng = G; c->nu = gr->nu; c->nv = gr->nv;
  c->na = na = gr->nu * gr->nv;
  c->dy = gr->dy; c->dz = gr->dz; c->u_max = gr->u_max; c->v_max = gr->v_max;
  c->ph = *ph;
  /* Reading (angular grid, Section 3.4): N unknowns per angle with zero
   * Dirichlet values one spacing beyond the outermost nodes, so the spacing
   * is 2 u_max / (N + 1) and the nodes sit symmetrically about 0. */
  c->du = 2.0 * gr->u_max / (gr->nu + 1);
  c->dv = 2.0 * gr->v_max / (gr->nv + 1);
  c->e_faces = (double *)malloc(sizeof(double) * (G + 1));
  c->e_c = (double *)malloc(sizeof(double) * G);
  c->de = (double *)malloc(sizeof(double) * G);
  c->s_face = (double *)malloc(sizeof(double) * (G + 1));
  c->s_base = (double *)malloc(sizeof(double) * (G + 1));
  c->t_face = (double *)calloc((size_t)G + 1, sizeof(double));
  c->ts = (double *)malloc(sizeof(double) * G);
  c->sig = (double *)malloc(sizeof(double) * G);
  c->p1 = (double *)calloc((size_t)G * G, sizeof(double));
  c->p2 = (double *)calloc((size_t)G * na * na, sizeof(double));
  c->u = (double *)malloc(sizeof(double) * gr->nu);
  c->v = (double *)malloc(sizeof(double) * gr->nv);
  for (int f = 0; f <= G; f++) c->e_faces[f] = gr->e_faces[f];
  for (int g = 0; g < G; g++) {
    c->de[g] = c->e_faces[g + 1] - c->e_faces[g];
    c->e_c[g] = 0.5 * (c->e_faces[g + 1] + c->e_faces[g]);
  }
  for (int i = 0; i < gr->nu; i++) c->u[i] = (i - 0.5 * (gr->nu - 1)) * c->du;
  for (int j = 0; j < gr->nv; j++) c->v[j] = (j - 0.5 * (gr->nv - 1)) * c->dv;

  /* Reading (energy floor): a face at E <= 0 has no finite Bragg-Kleeman
   * stopping power; it is evaluated at half the lowest group width instead.
   * The Bethe-Bloch tables hold their values below 0.5 MeV (where the
   * formula's logarithm loses its meaning). */
  double e_floor = 0.5 * c->de[0];
  if (ph->model == 1 && e_floor < 0.5) e_floor = 0.5;
  for (int f = 0; f <= G; f++) {
    double e = c->e_faces[f] > e_floor ? c->e_faces[f] : e_floor;
    c->s_base[f] = ph->model == 1 ? ph->s_scale * orc_bethe_water(ph, e) : bk_stopping(ph, e);
    /* Reading: the straggling formula is held below 0.5 MeV in both models
     * (at a few tens of keV its logarithm turns negative). */
    c->t_face[f] = ph->t_scale * orc_williams_water(ph, e > 0.5 ? e : 0.5);
  }
  fold_straggling(c);
  /* sigma_tr,g is the group average of the scattering coefficient
   * (after Eq. (0041-d)); here rho*sigma_tr is the Highland scattering power,
   * averaged exactly over [max(E_lo, floor), E_hi]. */
  for (int g = 0; g < G; g++) {
    double lo = c->e_faces[g] > e_floor ? c->e_faces[g] : e_floor;
    double hi = c->e_faces[g + 1];
    if (ph->model == 1) {
      /* group average by 8-point Gauss-Legendre (no closed-form primitive) */
      static const double x8[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                                   0.9602898564975363};
      static const double w8[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                                   0.1012285362903763};
      double acc = 0.0, mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
      for (int q = 0; q < 4; q++)
        acc += w8[q] * (orc_scat_power_water(ph, mid - half * x8[q]) + orc_scat_power_water(ph, mid + half * x8[q]));
      c->ts[g] = ph->ts_scale * 0.5 * acc;
    } else {
      c->ts[g] = ph->ts_scale * (highland_primitive(ph, hi) - highland_primitive(ph, lo)) / (hi - lo);
    }
    c->sig[g] = ph->sigma_ct;
  }
  /* P^1(g'->g) = lambda exp(-lambda (E_g' - E_g)) for g <= g' (protons only
   * lose energy), normalised so that each source group's probabilities over
   * the destination groups sum to one (particle conservation). */
  for (int gp = 0; gp < G; gp++) {
    double z = 0.0;
    for (int g = 0; g <= gp; g++) z += ph->lambda_p1 * exp(-ph->lambda_p1 * (c->e_c[gp] - c->e_c[g]));
    for (int g = 0; g <= gp; g++)
      c->p1[(size_t)gp * G + g] = ph->lambda_p1 * exp(-ph->lambda_p1 * (c->e_c[gp] - c->e_c[g])) / z;
  }
  /* P^2_g((u',v') -> (u,v)) = Gamma(theta; alpha, beta) / K with
   * theta = arccos Theta, Theta = (1 + u u' + v v') / (|(1,u,v)| |(1,u',v')|)
 * (the angle between the two directions);
   * K normalises the outgoing density: sum_a P^2 du dv = 1 for every a'. */
  for (int g = 0; g < G; g++) {
    for (int ap = 0; ap < na; ap++) {
      double up = c->u[ap % c->nu], vp = c->v[ap / c->nu];
      double k = 0.0;
      for (int a = 0; a < na; a++) {
        double uu = c->u[a % c->nu], vv = c->v[a / c->nu];
        /* theta = arccos(Theta), evaluated as atan2(|n x n'|, n . n') with
         * n = (1,u,v): the same angle, without the loss of accuracy of
         * arccos near theta = 0. */
        double cx = uu * vp - vv * up, cy = vv - vp, cz = up - uu;
        double th = atan2(sqrt(cx * cx + cy * cy + cz * cz), 1.0 + uu * up + vv * vp);
        double val = gamma_pdf(th, ph->g_alpha, ph->g_beta);
        c->p2[((size_t)g * na + a) * na + ap] = val;
        k += val * c->du * c->dv;
      }
      for (int a = 0; a < na; a++) c->p2[((size_t)g * na + a) * na + ap] /= (k > 0.0 ? k : 1.0);
    }
  }
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->e_faces); free(c->e_c); free(c->de); free(c->s_face); free(c->s_base); free(c->t_face); free(c->ts);
  free(c->sig); free(c->p1); free(c->p2); free(c->u); free(c->v);
  free(c);
}

/* Catastrophic removal cross section of every group, sig[g] (mass, cm^2/g),
 * in place of the constant of the physics parameters.  Section 4 writes the
 * removal term of group g with sigma_c,t,g, and sigma_c,s,g = sigma_c,t P^1 P^2
 * with sigma_c,t printed on the destination group.  Reading: a proton leaves
 * group g' at the rate of g' itself, so the removal term of group g uses
 * sig[g] and the source that group g receives from g' >= g uses sig[g'] (the
 * emitting group); only this form puts back into the next component exactly
 * what the removal took out (orc_source, orc_energy_blocks). */
void orc_set_sigma(orc_ctx *c, const double *sig) {
  for (int g = 0; g < c->ng; g++) c->sig[g] = sig[g];
}

void orc_get_tables(const orc_ctx *c, double *s_face, double *ts, double *sig, double *p1, double *p2,
                    double *u, double *v) {
  int G = c->ng, na = c->na;
  if (s_face) memcpy(s_face, c->s_face, sizeof(double) * (G + 1));
  if (ts) memcpy(ts, c->ts, sizeof(double) * G);
  if (sig) memcpy(sig, c->sig, sizeof(double) * G);
  if (p1) memcpy(p1, c->p1, sizeof(double) * G * G);
  if (p2) memcpy(p2, c->p2, sizeof(double) * G * na * na);
  if (u) memcpy(u, c->u, sizeof(double) * c->nu);
  if (v) memcpy(v, c->v, sizeof(double) * c->nv);
}

/* ------------------------------------------------------------------ */
/* Energy operator (Section 3.2, Eq. (0041-d) with T = 0)              */
/* ------------------------------------------------------------------ */

/* The 2x2 blocks of the semi-discrete energy operator for group g in a
 * medium of density rho:  d psi_g / dx = Agg psi_g + Aup psi_{g+1}.
 * Row 1 tests with phi^1/dE, row 2 with 3 phi^2/dE.  The interface value
 * at E_{g+1/2} is the upwind one from group g+1, psi^1_{g+1} - psi^2_{g+1}.
 * Reading (sign of the phi^2-tested lower-face flux): phi^2 = -1 at the
 * lower face, so [S psi phi^2] at E_{g-1/2} enters with a PLUS sign:
 *   + 3 S_- (psi^1_g - psi^2_g) / dE.
 * The printed minus sign would make a constant state with constant S drift. */
void orc_energy_blocks(const orc_ctx *c, int g, double rho, double agg[2][2], double aup[2][2]) {
  double a = rho / c->de[g];
  double sp = c->s_face[g + 1], sm = c->s_face[g];
  double sg = rho * c->sig[g];
  /* psi^1 row */
  agg[0][0] = -a * sm - sg;
  agg[0][1] = a * sm;
  /* psi^2 row: +3aS-(psi1 - psi2) - 3a(S+ + S-) psi1 - a(S+ - S-) psi2 - sigma psi2 */
  agg[1][0] = 3.0 * a * sm - 3.0 * a * (sp + sm);
  agg[1][1] = -3.0 * a * sm - a * (sp - sm) - sg;
  /* inflow from the group above: S+ (psi^1_{g+1} - psi^2_{g+1}) */
  if (g + 1 < c->ng) {
    aup[0][0] = a * sp;        aup[0][1] = -a * sp;
    aup[1][0] = 3.0 * a * sp;  aup[1][1] = -3.0 * a * sp;
  } else { /* nothing enters above the top face */
    aup[0][0] = aup[0][1] = aup[1][0] = aup[1][1] = 0.0;
  }
}

/* Apply the semi-discrete energy operator to one lane: out = A x.
 * x and out are [g][c] (2G values).  Stopping power (with the straggling
 * drift folded in) and removal only; the interior-penalty straggling part
 * is orc_straggle_apply. */
void orc_energy_apply(const orc_ctx *c, double rho, const double *x, double *out) {
  int G = c->ng;
  for (int g = 0; g < G; g++) {
    double agg[2][2], aup[2][2];
    orc_energy_blocks(c, g, rho, agg, aup);
    for (int r = 0; r < 2; r++) {
      double acc = agg[r][0] * x[2 * g] + agg[r][1] * x[2 * g + 1];
      if (g + 1 < G) acc += aup[r][0] * x[2 * g + 2] + aup[r][1] * x[2 * g + 3];
      out[2 * g + r] = acc;
    }
  }
}

/* Interior-penalty (SIPG) form of (rho/2) d/dE(T dpsi/dE) (Section 3.2, the
 * terms Q_1 and Q_2 of Eq. 0041-d), written out for the P1 basis
 * phi^1 = 1, phi^2 = 2 (E - E_g) / dE_g.  On group g, psi' = 2 psi^2 / dE_g
 * and, T being linear through its face values, int_g T = Tbar_g dE_g with
 * Tbar_g the mean of the two face values.  At an inner face f between
 * groups g (below) and g+1 (above):
 *   values   psi^- = psi^1_g + psi^2_g,  psi^+ = psi^1_{g+1} - psi^2_{g+1},
 *   jump     [psi] = psi^- - psi^+,
 *   average  {T psi'} = T_f (psi^2_g / dE_g + psi^2_{g+1} / dE_{g+1}),
 *   penalty  sigma_f = alpha T_f / h_f, alpha = (1 + 1)^2 / 2 = 2,
 *            h_f = (dE_g + dE_{g+1}) / 2.
 * The bilinear form is
 *   a(psi, v) = - sum_g int T psi' v' + sum_f ({T psi'}[v] + {T v'}[psi])
 *               - sum_f sigma_f [psi][v],
 * tested with v = phi^1_g / dE_g (row 1) and 3 phi^2_g / dE_g (row 2).
 * Reading (penalty): the printed penalty alpha [psi][phi] / dE carries
 * neither T nor a length; it is read as the standard sigma_f above.
 * Reading (outer faces): no diffusive flux through E_{1/2} and E_{G+1/2};
 * only inner faces carry the face terms, so straggling alone conserves the
 * particle count.  Rows of group g:
 *   row 1 = k/dE_g [ ({T psi'} - sigma [psi])_{g+1/2} - ({T psi'} - sigma [psi])_{g-1/2} ]
 *   row 2 = 3k/dE_g [ -4 Tbar_g psi^2_g / dE_g
 *                     + ({T psi'} + (T/dE_g - sigma)[psi])_{g+1/2}
 *                     + ({T psi'} + (T/dE_g - sigma)[psi])_{g-1/2} ],
 * k = rho / 2, a face term present only for inner faces.  The blocks:
 *   d psi_g / dx += alo psi_{g-1} + agg psi_g + aup psi_{g+1}. */
void orc_straggle_blocks(const orc_ctx *c, int g, double rho, double alo[2][2], double agg[2][2],
                         double aup[2][2]) {
  int G = c->ng;
  double k = 0.5 * rho, d = 1.0 / c->de[g];
  double tbar = 0.5 * (c->t_face[g] + c->t_face[g + 1]);
  for (int r = 0; r < 2; r++)
    for (int q = 0; q < 2; q++) alo[r][q] = agg[r][q] = aup[r][q] = 0.0;
  agg[1][1] = 3.0 * k * d * (-4.0 * tbar * d);
  if (g + 1 < G) { /* upper face: g is the lower side */
    double t = c->t_face[g + 1], du = 1.0 / c->de[g + 1];
    double sg = 2.0 * t / (0.5 * (c->de[g] + c->de[g + 1]));
    /* flux coefficients on (psi^2_g, psi^2_{g+1}); jump on (p1g, p2g, p1u, p2u) = (1, 1, -1, 1) */
    double w1 = k * d, w2 = 3.0 * k * d, tj = t * d - sg;
    agg[0][0] += w1 * (-sg);           agg[0][1] += w1 * (t * d - sg);
    aup[0][0] += w1 * sg;              aup[0][1] += w1 * (t * du - sg);
    agg[1][0] += w2 * tj;              agg[1][1] += w2 * (t * d + tj);
    aup[1][0] += w2 * (-tj);           aup[1][1] += w2 * (t * du + tj);
  }
  if (g > 0) { /* lower face: g is the upper side */
    double t = c->t_face[g], dl = 1.0 / c->de[g - 1];
    double sg = 2.0 * t / (0.5 * (c->de[g] + c->de[g - 1]));
    /* flux on (psi^2_{g-1}, psi^2_g); jump on (p1l, p2l, p1g, p2g) = (1, 1, -1, 1) */
    double w1 = -k * d, w2 = 3.0 * k * d, tj = t * d - sg;
    alo[0][0] += w1 * (-sg);           alo[0][1] += w1 * (t * dl - sg);
    agg[0][0] += w1 * sg;              agg[0][1] += w1 * (t * d - sg);
    alo[1][0] += w2 * tj;              alo[1][1] += w2 * (t * dl + tj);
    agg[1][0] += w2 * (-tj);           agg[1][1] += w2 * (t * d + tj);
  }
}

/* out = A_T x for one lane, A_T the interior-penalty straggling operator. */
void orc_straggle_apply(const orc_ctx *c, double rho, const double *x, double *out) {
  int G = c->ng;
  for (int g = 0; g < G; g++) {
    double alo[2][2], agg[2][2], aup[2][2];
    orc_straggle_blocks(c, g, rho, alo, agg, aup);
    for (int r = 0; r < 2; r++) {
      double acc = agg[r][0] * x[2 * g] + agg[r][1] * x[2 * g + 1];
      if (g > 0) acc += alo[r][0] * x[2 * g - 2] + alo[r][1] * x[2 * g - 1];
      if (g + 1 < G) acc += aup[r][0] * x[2 * g + 2] + aup[r][1] * x[2 * g + 3];
      out[2 * g + r] = acc;
    }
  }
}

/* Energy content per unit (u,v,y,z) of a DG state:  int E psi dE =
 *   sum_g dE_g (E_g psi^1_g + dE_g psi^2_g / 6). */
static double energy_content(const orc_ctx *c, const double *x) {
  double s = 0.0;
  for (int g = 0; g < c->ng; g++) s += c->de[g] * (c->e_c[g] * x[2 * g] + c->de[g] * x[2 * g + 1] / 6.0);
  return s;
}

static void inv2(const double m[2][2], double out[2][2]) {
  double det = m[0][0] * m[1][1] - m[0][1] * m[1][0];
  out[0][0] = m[1][1] / det;  out[0][1] = -m[0][1] / det;
  out[1][0] = -m[1][0] / det; out[1][1] = m[0][0] / det;
}

/* One Crank-Nicolson step of length h for one lane:
 *   (I - h/2 A) x_new = (I + h/2 A) x_old + h/2 (src_old + src_new),
 * where src_sum = src_old + src_new acts on psi^1 only (Remark 1).
 * A = A_S (stopping, drift, removal; block upper-bidiagonal) + A_T
 * (interior-penalty straggling; block tridiagonal).
 *  * Without straggling, or with it explicit (orc_set_straggling_cn 0):
 *      (I - h/2 A_S) x_new = (I + h/2 A_S) x_old + h A_T x_old + h/2 src,
 *    solved from the top group down (x_{G+1} = 0):
 *      M_g x_g = rhs_g + h/2 Aup x_{g+1}.
 *    This follows the authors' remark (kept in the paper's source, after
 *    the splitting section) that the small straggling term is taken
 *    explicitly in the implicit half of CN.
 *  * With full CN (orc_set_straggling_cn 1) the system is block
 *    tridiagonal and is solved by block elimination from the top group down
 *    and substitution upward.
 * Returns the deposited energy content of the lane (difference form) and,
 * through *edep_w, the same quantity from the operator form
 *   -(h/2) phi^T A_S (x_old + x_new) - h phi^T A_T x_old - (h/2) phi^T src
 * (full CN: -(h/2) phi^T A (x_old + x_new) - (h/2) phi^T src). */
double orc_energy_cn_lane(const orc_ctx *c, double rho, double h, double *x, const double *src_sum,
                          double *edep_w) {
  int G = c->ng;
  int strag = c->strag_on, full = strag && c->strag_cn;
  double *old = (double *)malloc(sizeof(double) * 2 * G);
  double *ax = (double *)malloc(sizeof(double) * 2 * G);
  double *tx = (double *)malloc(sizeof(double) * 2 * G);
  double *rhs = (double *)malloc(sizeof(double) * 2 * G);
  double *dp = full ? (double *)malloc(sizeof(double) * 4 * G) : NULL; /* eliminated diagonal blocks */
  double hh = 0.5 * h;
  memcpy(old, x, sizeof(double) * 2 * G);
  orc_energy_apply(c, rho, old, ax);
  if (strag) orc_straggle_apply(c, rho, old, tx);
  for (int k = 0; k < 2 * G; k++) rhs[k] = old[k] + hh * ax[k] + (strag ? (full ? hh : h) * tx[k] : 0.0);
  if (src_sum)
    for (int g = 0; g < G; g++) rhs[2 * g] += hh * src_sum[g];
  if (!full) {
    for (int g = G - 1; g >= 0; g--) {
      double agg[2][2], aup[2][2], m[2][2], b[2];
      orc_energy_blocks(c, g, rho, agg, aup);
      b[0] = rhs[2 * g];
      b[1] = rhs[2 * g + 1];
      if (g + 1 < G) {
        b[0] += hh * (aup[0][0] * x[2 * g + 2] + aup[0][1] * x[2 * g + 3]);
        b[1] += hh * (aup[1][0] * x[2 * g + 2] + aup[1][1] * x[2 * g + 3]);
      }
      m[0][0] = 1.0 - hh * agg[0][0]; m[0][1] = -hh * agg[0][1];
      m[1][0] = -hh * agg[1][0];      m[1][1] = 1.0 - hh * agg[1][1];
      double det = m[0][0] * m[1][1] - m[0][1] * m[1][0];
      x[2 * g] = (m[1][1] * b[0] - m[0][1] * b[1]) / det;
      x[2 * g + 1] = (-m[1][0] * b[0] + m[0][0] * b[1]) / det;
    }
  } else {
    /* rows: L_g x_{g-1} + D_g x_g + U_g x_{g+1} = rhs_g with
     * D = I - hh (A_S,gg + A_T,gg), U = -hh (A_S,up + A_T,up), L = -hh A_T,lo.
     * Eliminate from the top: D'_g = D_g - U_g D'^{-1}_{g+1} L_{g+1},
     * b'_g = b_g - U_g D'^{-1}_{g+1} b'_{g+1}; then x_0 = D'^{-1}_0 b'_0 and
     * x_g = D'^{-1}_g (b'_g - L_g x_{g-1}) upward. */
    double lnext[2][2] = {{0, 0}, {0, 0}};
    for (int g = G - 1; g >= 0; g--) {
      double sgg[2][2], sup[2][2], tlo[2][2], tgg[2][2], tup[2][2], D[2][2], U[2][2], Di[2][2];
      orc_energy_blocks(c, g, rho, sgg, sup);
      orc_straggle_blocks(c, g, rho, tlo, tgg, tup);
      for (int r = 0; r < 2; r++)
        for (int q = 0; q < 2; q++) {
          D[r][q] = (r == q ? 1.0 : 0.0) - hh * (sgg[r][q] + tgg[r][q]);
          U[r][q] = (g + 1 < G) ? -hh * (sup[r][q] + tup[r][q]) : 0.0;
        }
      if (g + 1 < G) {
        /* W = U_g D'^{-1}_{g+1} */
        double Dn[2][2], W[2][2];
        for (int r = 0; r < 2; r++)
          for (int q = 0; q < 2; q++) Dn[r][q] = dp[4 * (g + 1) + 2 * r + q];
        inv2(Dn, Di);
        for (int r = 0; r < 2; r++)
          for (int q = 0; q < 2; q++) W[r][q] = U[r][0] * Di[0][q] + U[r][1] * Di[1][q];
        for (int r = 0; r < 2; r++) {
          for (int q = 0; q < 2; q++) D[r][q] -= W[r][0] * lnext[0][q] + W[r][1] * lnext[1][q];
        }
        double b0 = rhs[2 * g] - (W[0][0] * rhs[2 * g + 2] + W[0][1] * rhs[2 * g + 3]);
        double b1 = rhs[2 * g + 1] - (W[1][0] * rhs[2 * g + 2] + W[1][1] * rhs[2 * g + 3]);
        rhs[2 * g] = b0;
        rhs[2 * g + 1] = b1;
      }
      for (int r = 0; r < 2; r++)
        for (int q = 0; q < 2; q++) {
          dp[4 * g + 2 * r + q] = D[r][q];
          lnext[r][q] = (g > 0) ? -hh * tlo[r][q] : 0.0;
        }
    }
    for (int g = 0; g < G; g++) {
      double tlo[2][2], tgg[2][2], tup[2][2], Dg[2][2], Di[2][2], b0 = rhs[2 * g], b1 = rhs[2 * g + 1];
      if (g > 0) {
        orc_straggle_blocks(c, g, rho, tlo, tgg, tup);
        b0 -= -hh * (tlo[0][0] * x[2 * g - 2] + tlo[0][1] * x[2 * g - 1]);
        b1 -= -hh * (tlo[1][0] * x[2 * g - 2] + tlo[1][1] * x[2 * g - 1]);
      }
      for (int r = 0; r < 2; r++)
        for (int q = 0; q < 2; q++) Dg[r][q] = dp[4 * g + 2 * r + q];
      inv2(Dg, Di);
      x[2 * g] = Di[0][0] * b0 + Di[0][1] * b1;
      x[2 * g + 1] = Di[1][0] * b0 + Di[1][1] * b1;
    }
  }
  double dep = energy_content(c, old) - energy_content(c, x);
  if (edep_w) {
    double *sum = rhs; /* reuse */
    for (int k = 0; k < 2 * G; k++) sum[k] = old[k] + x[k];
    orc_energy_apply(c, rho, sum, ax);
    double w = -hh * energy_content(c, ax);
    if (strag) {
      orc_straggle_apply(c, rho, full ? sum : old, tx);
      w -= (full ? hh : h) * energy_content(c, tx);
    }
    if (src_sum) {
      double s = 0.0;
      for (int g = 0; g < G; g++) s += c->de[g] * c->e_c[g] * src_sum[g];
      w -= hh * s;
    }
    *edep_w = w;
  }
  free(old); free(ax); free(tx); free(rhs); free(dp);
  return dep;
}

/* Energy substep E(h) for every lane (y,z,u,v) of one component (Remark 2:
 * independent lanes).  psi is one component [g][c][a][p][q]; src_sum is
 * [g][a][p][q] or NULL; rho_yz is [p][q].  Deposited energy per lateral cell
 * (MeV per source proton, i.e. already multiplied by du dv dy dz) is added to
 * edep_yz[p][q] and edep_w_yz (operator form) when those are non-NULL. */
void orc_energy_substep(const orc_ctx *c, double h, const double *rho_yz, double *psi, const double *src_sum,
                        double *edep_yz, double *edep_w_yz) {
  int G = c->ng, na = c->na, ny = c->ny, nz = c->nz;
  double cellw = c->du * c->dv * c->dy * c->dz;
#pragma omp parallel for schedule(static)
  for (int pq = 0; pq < ny * nz; pq++) {
    int p = pq / nz, q = pq % nz;
    double *x = (double *)malloc(sizeof(double) * 2 * G);
    double *s = src_sum ? (double *)malloc(sizeof(double) * G) : NULL;
    double dep = 0.0, depw = 0.0;
    for (int a = 0; a < na; a++) {
      for (int g = 0; g < G; g++) {
        x[2 * g] = psi[IDX5(c, g, 0, a, p, q)];
        x[2 * g + 1] = psi[IDX5(c, g, 1, a, p, q)];
        if (s) s[g] = src_sum[(((size_t)g * na + a) * ny + p) * nz + q];
      }
      double w = 0.0;
      dep += orc_energy_cn_lane(c, rho_yz[pq], h, x, s, &w);
      depw += w;
      for (int g = 0; g < G; g++) {
        psi[IDX5(c, g, 0, a, p, q)] = x[2 * g];
        psi[IDX5(c, g, 1, a, p, q)] = x[2 * g + 1];
      }
    }
    if (edep_yz) edep_yz[pq] += dep * cellw;
    if (edep_w_yz) edep_w_yz[pq] += depw * cellw;
    free(x); free(s);
  }
}

/* ------------------------------------------------------------------ */
/* Catastrophic source (Remark 1, Section 4, Appendix A.4)              */
/* ------------------------------------------------------------------ */

/* src^1_g(a) = du dv sum_{a'} sum_{g' >= g} sigma_{c,s,g'->g}(a'->a)
 *              psi^1_{g'}(a') dE_{g'} / dE_g,
 * with sigma_{c,s,g'->g}(a'->a) = rho sigma_{c,t,g'} P^1(g'->g) P^2_g(a'->a).
 * Reading: the removal rate is the source group's sigma_{c,t,g'}.
 * prev is the previous component [g][c][a][p][q]; out is [g][a][p][q]. */
void orc_source(const orc_ctx *c, const double *rho_yz, const double *prev, double *out) {
  int G = c->ng, na = c->na, ny = c->ny, nz = c->nz;
#pragma omp parallel for schedule(static)
  for (int pq = 0; pq < ny * nz; pq++) {
    int p = pq / nz, q = pq % nz;
    double rho = rho_yz[pq];
    double *r = (double *)malloc(sizeof(double) * na);
    for (int g = 0; g < G; g++) {
      /* the energy sum first: r(a') = sum_{g' >= g} rho sigma_g' P^1(g'->g) psi^1_g'(a') dE_g' / dE_g */
      for (int ap = 0; ap < na; ap++) {
        double inner = 0.0;
        for (int gp = g; gp < G; gp++)
          inner += rho * c->sig[gp] * c->p1[(size_t)gp * G + g] * prev[IDX5(c, gp, 0, ap, p, q)] * c->de[gp] / c->de[g];
        r[ap] = inner;
      }
      /* then the angle sum with P^2_g */
      for (int a = 0; a < na; a++) {
        double acc = 0.0;
        for (int ap = 0; ap < na; ap++) acc += c->p2[((size_t)g * na + a) * na + ap] * r[ap];
        out[(((size_t)g * na + a) * ny + p) * nz + q] = c->du * c->dv * acc;
      }
    }
    free(r);
  }
}

/* ------------------------------------------------------------------ */
/* Lateral transport (Section 3.4, Eq. (distansport), Remark 3)         */
/* ------------------------------------------------------------------ */

/* Slope limiter eta(theta) = max[0, min(2 theta, 1), min(theta, 2)]. */
static double eta_limiter(double th) {
  double a = fmin(2.0 * th, 1.0), b = fmin(th, 2.0);
  double m = a > b ? a : b;
  return m > 0.0 ? m : 0.0;
}

/* Limited slope delta = (psi_{p+1} - psi_p) eta(theta), theta = num / (psi_{p+1} - psi_p).
 * Where psi_{p+1} = psi_p the slope is zero whatever eta (eta <= 2). */
static double limited_slope(double num, double den) {
  if (den == 0.0) return 0.0;
  return den * eta_limiter(num / den);
}

/* Numerical flux through the face between cells m (left) and m+1 (right)
 * along one line of values f[] with zero ghost cells outside 0..n-1:
 *   Psi = s+ psi^L - s- psi^R,
 *   psi^L = psi_m + delta^L / 2,      theta^L = (psi_m - psi_{m-1}) / (psi_{m+1} - psi_m),
 *   psi^R = psi_{m+1} - delta^R / 2,  theta^R = (psi_{m+2} - psi_{m+1}) / (psi_{m+1} - psi_m).
 * Reading: the paper prints theta only for the left state; the right state
 * uses the mirrored ratio, as in the flux-limiter form it cites. */
static double face_flux(const double *f, int n, long stride, int m, double s) {
#define VAL(k) (((k) >= 0 && (k) < n) ? f[(long)(k) * stride] : 0.0)
  double pm1 = VAL(m - 1), p0 = VAL(m), p1 = VAL(m + 1), p2 = VAL(m + 2);
#undef VAL
  double sp = s > 0.0 ? s : 0.0, sm = s < 0.0 ? -s : 0.0;
  double flux = 0.0;
  if (sp > 0.0) flux += sp * (p0 + 0.5 * limited_slope(p0 - pm1, p1 - p0));
  if (sm > 0.0) flux -= sm * (p1 - 0.5 * limited_slope(p2 - p1, p1 - p0));
  return flux;
}

/* Semi-discrete right-hand side L(psi) = -(F_{p+1/2} - F_{p-1/2})/dy
 *                                        - (G_{q+1/2} - G_{q-1/2})/dz
 * for one (y,z) plane moving with angle (uu, vv). */
static void transport_rhs(const orc_ctx *c, double uu, double vv, const double *f, double *out) {
  int ny = c->ny, nz = c->nz;
  for (int p = 0; p < ny; p++)
    for (int q = 0; q < nz; q++) {
      const double *col = f + q;            /* line along y at fixed q */
      const double *row = f + (long)p * nz; /* line along z at fixed p */
      double fy = face_flux(col, ny, nz, p, uu) - face_flux(col, ny, nz, p - 1, uu);
      double fz = face_flux(row, nz, 1, q, vv) - face_flux(row, nz, 1, q - 1, vv);
      out[(long)p * nz + q] = -fy / c->dy - fz / c->dz;
    }
}

/* The first-order upwind part of the same operator: the fluxes without
 * their slope terms, s+ psi_m - s- psi_{m+1}. */
static void transport_rhs_upwind(const orc_ctx *c, double uu, double vv, const double *f, double *out) {
  int ny = c->ny, nz = c->nz;
#define V(p, q) (((p) >= 0 && (p) < ny && (q) >= 0 && (q) < nz) ? f[(long)(p) * nz + (q)] : 0.0)
  double up = uu > 0.0 ? uu : 0.0, um = uu < 0.0 ? -uu : 0.0;
  double vp = vv > 0.0 ? vv : 0.0, vm = vv < 0.0 ? -vv : 0.0;
  for (int p = 0; p < ny; p++)
    for (int q = 0; q < nz; q++) {
      double fy = (up * V(p, q) - um * V(p + 1, q)) - (up * V(p - 1, q) - um * V(p, q));
      double fz = (vp * V(p, q) - vm * V(p, q + 1)) - (vp * V(p, q - 1) - vm * V(p, q));
      out[(long)p * nz + q] = -fy / c->dy - fz / c->dz;
    }
#undef V
}

/* L(psi) (first_order = 0) or its first-order upwind part L1 (1) for one
 * plane [p][q] moving with angle (uu, vv). */
void orc_transport_apply(const orc_ctx *c, double uu, double vv, const double *f, double *out, int first_order) {
  if (first_order) transport_rhs_upwind(c, uu, vv, f, out);
  else transport_rhs(c, uu, vv, f, out);
}

/* Transport time integrator (Remark 3).  0 (default): the slope is treated
 * explicitly, which makes the Crank-Nicolson average an explicit trapezoid
 * (Heun).  1: Crank-Nicolson in which only the slope part of the implicit
 * half is taken from the old state (the remark's "slope explicitly in the
 * implicit part"); the first-order upwind part stays implicit and is solved
 * by one sweep in the upwind direction. */
void orc_set_transport_cn(orc_ctx *c, int cn) { c->transport_cn = cn != 0; }

/* Transport substep T(h) for every (g, c, u, v) plane (Remark 2).
 *  * Heun: psi* = psi + h L(psi),  psi_new = psi + h/2 (L(psi) + L(psi*)).
 *  * CN with lagged slope: with L = L1 + Ld (upwind part, slope part),
 *      psi_new - psi = h/2 (L(psi) + L1(psi_new) + Ld(psi)),
 *    i.e. (I - h/2 L1) psi_new = psi + h/2 L(psi) + h/2 Ld(psi).
 *    I - h/2 L1 couples a cell only to its upstream neighbours in y and z
 *    (zero inflow outside the plane), so visiting the cells in the upwind
 *    order solves it exactly:
 *      psi_new(p,q) = (r(p,q) + cy psi_new(p-sy,q) + cz psi_new(p,q-sz)) / (1 + cy + cz),
 *    cy = h |u| / (2 dy), cz = h |v| / (2 dz), sy, sz the signs of u, v. */
void orc_transport_substep(const orc_ctx *c, double h, double *psi) {
  int G = c->ng, na = c->na, n = c->ny * c->nz, ny = c->ny, nz = c->nz;
  int cn = c->transport_cn;
#pragma omp parallel for schedule(static)
  for (int plane = 0; plane < G * 2 * na; plane++) {
    int a = plane % na;
    double uu = c->u[a % c->nu], vv = c->v[a / c->nu];
    double *f = psi + (size_t)plane * n;
    double *l0 = (double *)malloc(sizeof(double) * n);
    double *st = (double *)malloc(sizeof(double) * n);
    double *l1 = (double *)malloc(sizeof(double) * n);
    transport_rhs(c, uu, vv, f, l0);
    if (!cn) {
      for (int k = 0; k < n; k++) st[k] = f[k] + h * l0[k];
      transport_rhs(c, uu, vv, st, l1);
      for (int k = 0; k < n; k++) f[k] = f[k] + 0.5 * h * (l0[k] + l1[k]);
    } else {
      transport_rhs_upwind(c, uu, vv, f, l1);
      /* r = psi + h/2 L + h/2 (L - L1) */
      for (int k = 0; k < n; k++) st[k] = f[k] + 0.5 * h * l0[k] + 0.5 * h * (l0[k] - l1[k]);
      double cy = 0.5 * h * fabs(uu) / c->dy, cz = 0.5 * h * fabs(vv) / c->dz;
      int sy = uu < 0.0 ? -1 : 1, sz = vv < 0.0 ? -1 : 1;
      for (int i = 0; i < ny; i++) {
        int p = sy > 0 ? i : ny - 1 - i;
        for (int j = 0; j < nz; j++) {
          int q = sz > 0 ? j : nz - 1 - j;
          int pu = p - sy, qu = q - sz;
          double xy = (pu >= 0 && pu < ny) ? f[(long)pu * nz + q] : 0.0; /* already new */
          double xz = (qu >= 0 && qu < nz) ? f[(long)p * nz + qu] : 0.0;
          f[(long)p * nz + q] = (st[(long)p * nz + q] + cy * xy + cz * xz) / (1.0 + cy + cz);
        }
      }
    }
    free(l0); free(st); free(l1);
  }
}

/* ------------------------------------------------------------------ */
/* Angular diffusion (Section 3.4, Eqs. (sd), (fly))                   */
/* ------------------------------------------------------------------ */

/* Angular substep A(h) for every (g, c, y, z) slab (Remark 2).  The
 * five-point Laplacian with zero Dirichlet values is diagonalised by the
 * discrete sine transform; each mode (m,n) has eigenvalue
 *   lam = (2cos(pi m/(Nu+1)) - 2)/du^2 + (2cos(pi n/(Nv+1)) - 2)/dv^2
 * and Crank-Nicolson with coefficient kappa/2, kappa = rho sigma_tr,g,
 * multiplies it by r = (1 + h kappa lam / 4) / (1 - h kappa lam / 4).
 * The transform is written as explicit sine sums (one direction at a time)
 * with the orthonormal scaling sqrt(2/(N+1)) in each direction (the paper's
 * 1/(IJ) inverse scaling with I = N+1 is the same map). */
void orc_angular_substep(const orc_ctx *c, double h, const double *rho_yz, double *psi) {
  int G = c->ng, nu = c->nu, nv = c->nv, na = c->na, ny = c->ny, nz = c->nz;
  double *su = (double *)malloc(sizeof(double) * nu * nu);
  double *sv = (double *)malloc(sizeof(double) * nv * nv);
  double *lam = (double *)malloc(sizeof(double) * na);
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < nu; m++)
    for (int i = 0; i < nu; i++) su[m * nu + i] = sqrt(2.0 / (nu + 1)) * sin(pi * (m + 1) * (i + 1) / (nu + 1));
  for (int n = 0; n < nv; n++)
    for (int j = 0; j < nv; j++) sv[n * nv + j] = sqrt(2.0 / (nv + 1)) * sin(pi * (n + 1) * (j + 1) / (nv + 1));
  for (int n = 0; n < nv; n++)
    for (int m = 0; m < nu; m++)
      lam[n * nu + m] = (2.0 * cos(pi * (m + 1) / (nu + 1)) - 2.0) / (c->du * c->du) +
                        (2.0 * cos(pi * (n + 1) / (nv + 1)) - 2.0) / (c->dv * c->dv);
#pragma omp parallel for schedule(static)
  for (long slab = 0; slab < (long)G * 2 * ny * nz; slab++) {
    long gc = slab / ((long)ny * nz);
    int pq = (int)(slab % ((long)ny * nz));
    int g = (int)(gc / 2);
    double kappa = rho_yz[pq] * c->ts[g];
    double *base = psi + (size_t)gc * na * ny * nz + pq;
    long st = (long)ny * nz; /* stride between angles */
    double *x = (double *)malloc(sizeof(double) * na);
    double *t = (double *)malloc(sizeof(double) * na);
    double *w = (double *)malloc(sizeof(double) * na);
    for (int a = 0; a < na; a++) x[a] = base[a * st];
    /* The 2-D sine basis of Eq. (fly) is a product sin(.i) sin(.j), so each
     * 2-D sum is done as a sum over i followed by a sum over j.
     * forward: w[j][m] = sum_i su[m][i] x[j][i];  t[n][m] = sum_j sv[n][j] w[j][m] */
    for (int j = 0; j < nv; j++)
      for (int m = 0; m < nu; m++) {
        double acc = 0.0;
        for (int i = 0; i < nu; i++) acc += su[m * nu + i] * x[j * nu + i];
        w[j * nu + m] = acc;
      }
    for (int n = 0; n < nv; n++)
      for (int m = 0; m < nu; m++) {
        double acc = 0.0;
        for (int j = 0; j < nv; j++) acc += sv[n * nv + j] * w[j * nu + m];
        double q = 0.25 * h * kappa * lam[n * nu + m];
        t[n * nu + m] = acc * (c->angular_exact ? exp(2.0 * q) : (1.0 + q) / (1.0 - q));
      }
    /* inverse (the orthonormal DST-I is its own inverse), same two sums */
    for (int j = 0; j < nv; j++)
      for (int m = 0; m < nu; m++) {
        double acc = 0.0;
        for (int n = 0; n < nv; n++) acc += sv[n * nv + j] * t[n * nu + m];
        w[j * nu + m] = acc;
      }
    for (int j = 0; j < nv; j++)
      for (int i = 0; i < nu; i++) {
        double acc = 0.0;
        for (int m = 0; m < nu; m++) acc += su[m * nu + i] * w[j * nu + m];
        x[j * nu + i] = acc;
      }
    for (int a = 0; a < na; a++) base[a * st] = x[a];
    free(x); free(t); free(w);
  }
  free(su); free(sv); free(lam);
}

/* ------------------------------------------------------------------ */
/* Beam (Section 4, Eq. (bdy))                                          */
/* ------------------------------------------------------------------ */

static double std_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }
static double std_pdf(double x) { return exp(-0.5 * x * x) / sqrt(2.0 * 3.14159265358979323846); }

/* Probability mass of N(mu, s^2) in [lo, hi]. */
static double gauss_mass(double lo, double hi, double mu, double s) {
  double a = (lo - mu) / s, b = (hi - mu) / s;
  if (a > 0.0) return std_cdf(-a) - std_cdf(-b); /* upper tail: avoid 1 - 1 */
  return std_cdf(b) - std_cdf(a);
}

/* psi_p(x=0): the Gaussian of Eq. (bdy) projected on the discrete space.
 * Lateral: cell averages.  Angle: average over each node's cell of width
 * du (Reading: with sigma_u = 1e-6 the beam is narrower than one node, and
 * the cell average splits it evenly between the nodes next to u0).
 * Energy: DG L2 projection, psi^1 = (1/dE) int f, psi^2 = (3/dE) int f phi^2.
 * The constant C is fixed by sum psi^1 dE du dv dy dz = 1 (one proton). */
void orc_init_beam(const orc_ctx *c, const orc_beam *b, double *psi) {
  int G = c->ng, nu = c->nu, nv = c->nv, na = c->na, ny = c->ny, nz = c->nz;
  double *ey = (double *)malloc(sizeof(double) * 2 * G);
  double *ay = (double *)malloc(sizeof(double) * na);
  double *yy = (double *)malloc(sizeof(double) * ny);
  double *zz = (double *)malloc(sizeof(double) * nz);
  double tot_e = 0.0, tot_a = 0.0, tot_y = 0.0, tot_z = 0.0;
  for (int g = 0; g < G; g++) {
    double lo = c->e_faces[g], hi = c->e_faces[g + 1], de = c->de[g];
    double m0 = gauss_mass(lo, hi, b->e0, b->sigma_e);
    double al = (lo - b->e0) / b->sigma_e, be = (hi - b->e0) / b->sigma_e;
    double m1 = b->sigma_e * (std_pdf(al) - std_pdf(be)) + (b->e0 - c->e_c[g]) * m0; /* int (E-E_g) f */
    ey[2 * g] = m0 / de;
    ey[2 * g + 1] = 3.0 / de * (2.0 / de) * m1;
    tot_e += ey[2 * g] * de;
  }
  for (int j = 0; j < nv; j++)
    for (int i = 0; i < nu; i++) {
      double mu = gauss_mass(c->u[i] - 0.5 * c->du, c->u[i] + 0.5 * c->du, b->u0, b->sigma_u) / c->du;
      double mv = gauss_mass(c->v[j] - 0.5 * c->dv, c->v[j] + 0.5 * c->dv, b->v0, b->sigma_v) / c->dv;
      ay[j * nu + i] = mu * mv;
      tot_a += mu * mv * c->du * c->dv;
    }
  for (int p = 0; p < ny; p++) {
    double lo = (p - 0.5 * ny) * c->dy, hi = (p + 1 - 0.5 * ny) * c->dy;
    yy[p] = gauss_mass(lo, hi, b->y0, b->sigma_y) / c->dy;
    tot_y += yy[p] * c->dy;
  }
  for (int q = 0; q < nz; q++) {
    double lo = (q - 0.5 * nz) * c->dz, hi = (q + 1 - 0.5 * nz) * c->dz;
    zz[q] = gauss_mass(lo, hi, b->z0, b->sigma_z) / c->dz;
    tot_z += zz[q] * c->dz;
  }
  double norm = 1.0 / (tot_e * tot_a * tot_y * tot_z);
  for (int g = 0; g < G; g++)
    for (int cc = 0; cc < 2; cc++)
      for (int a = 0; a < na; a++)
        for (int p = 0; p < ny; p++)
          for (int q = 0; q < nz; q++)
            psi[IDX5(c, g, cc, a, p, q)] = norm * ey[2 * g + cc] * ay[a] * yy[p] * zz[q];
  free(ey); free(ay); free(yy); free(zz);
}

/* ------------------------------------------------------------------ */
/* Depth march (Sections 3.1 and 3.3)                                   */
/* ------------------------------------------------------------------ */

/* Energy substep of length h for all components in lock-step.  The source
 * of component k (k >= 1) is the catastrophic source of component k-1,
 * evaluated at the start and at the end of the same substep (trapezoid). */
static void energy_all(const orc_ctx *c, const orc_march_opts *o, double h, const double *rho_yz, double *psi,
                       double *edep_yz, double *edep_w_yz, double *srcA, double *srcB) {
  size_t ncomp = (size_t)c->ng * 2 * c->na * c->ny * c->nz;
  size_t nsrc = (size_t)c->ng * c->na * c->ny * c->nz;
  for (int k = 0; k <= o->n_scatter; k++) {
    double *pk = psi + (size_t)k * ncomp;
    const double *src = NULL;
    if (k >= 1) src = srcB; /* holds src(psi_{k-1}, old) + src(psi_{k-1}, new) */
    if (k < o->n_scatter) orc_source(c, rho_yz, pk, srcA); /* source for k+1 from the old state */
    orc_energy_substep(c, h, rho_yz, pk, src, edep_yz, edep_w_yz);
    if (k < o->n_scatter) {
      double *tmp = (double *)malloc(sizeof(double) * nsrc);
      orc_source(c, rho_yz, pk, tmp); /* ... and from the new state */
      for (size_t e = 0; e < nsrc; e++) srcB[e] = srcA[e] + tmp[e];
      free(tmp);
    }
  }
}

int orc_march(const orc_ctx *c, const orc_march_opts *o, const orc_beam *b, const double *rho, int n_steps,
              double dx, double *psi, double *dose, double *edep_w, double *fluence) {
  int ny = c->ny, nz = c->nz, ncomp_k = o->n_scatter + 1;
  size_t ncomp = (size_t)c->ng * 2 * c->na * ny * nz;
  size_t nsrc = (size_t)c->ng * c->na * ny * nz;
  double *srcA = o->n_scatter > 0 ? (double *)calloc(nsrc, sizeof(double)) : NULL;
  double *srcB = o->n_scatter > 0 ? (double *)calloc(nsrc, sizeof(double)) : NULL;
  double *edep = (double *)calloc((size_t)ny * nz, sizeof(double));
  double *edw = (double *)calloc((size_t)ny * nz, sizeof(double));
  if (b) {
    memset(psi, 0, sizeof(double) * ncomp * ncomp_k);
    orc_init_beam(c, b, psi);
  }
  if (fluence) orc_fluence(c, psi, ncomp_k, fluence);
  for (int s = 0; s < n_steps; s++) {
    const double *rho_yz = rho + (size_t)s * ny * nz;
    memset(edep, 0, sizeof(double) * ny * nz);
    memset(edw, 0, sizeof(double) * ny * nz);
    if (o->scheme == 0) {
      /* Strang: E(h/2) T(h/2) A(h) T(h/2) E(h/2), CN in each substep */
      if (o->do_energy) energy_all(c, o, 0.5 * dx, rho_yz, psi, edep, edw, srcA, srcB);
      if (o->do_transport)
        for (int k = 0; k < ncomp_k; k++) orc_transport_substep(c, 0.5 * dx, psi + k * ncomp);
      if (o->do_angular)
        for (int k = 0; k < ncomp_k; k++) orc_angular_substep(c, dx, rho_yz, psi + k * ncomp);
      if (o->do_transport)
        for (int k = 0; k < ncomp_k; k++) orc_transport_substep(c, 0.5 * dx, psi + k * ncomp);
      if (o->do_energy) energy_all(c, o, 0.5 * dx, rho_yz, psi, edep, edw, srcA, srcB);
    } else {
      /* first-order (Lie) splitting: E(h) T(h) A(h), Eqs. (split-1..3) */
      if (o->do_energy) energy_all(c, o, dx, rho_yz, psi, edep, edw, srcA, srcB);
      if (o->do_transport)
        for (int k = 0; k < ncomp_k; k++) orc_transport_substep(c, dx, psi + k * ncomp);
      if (o->do_angular)
        for (int k = 0; k < ncomp_k; k++) orc_angular_substep(c, dx, rho_yz, psi + k * ncomp);
    }
    /* D = E_dep / rho per unit volume (Eq. (en_d) and the definition above it) */
    for (int pq = 0; pq < ny * nz; pq++) {
      double m = rho_yz[pq] * dx * c->dy * c->dz;
      if (dose) dose[(size_t)s * ny * nz + pq] = m > 0.0 ? edep[pq] / m : 0.0;
      if (edep_w) edep_w[(size_t)s * ny * nz + pq] = m > 0.0 ? edw[pq] / m : 0.0;
    }
    if (fluence) orc_fluence(c, psi, ncomp_k, fluence + (size_t)(s + 1) * ny * nz);
  }
  free(srcA); free(srcB); free(edep); free(edw);
  return 0;
}

/* Planar fluence per lateral cell: du dv sum_{k,g,a} psi^1 dE (protons/cm^2). */
void orc_fluence(const orc_ctx *c, const double *psi, int ncomp_k, double *out) {
  int ny = c->ny, nz = c->nz;
  size_t ncomp = (size_t)c->ng * 2 * c->na * ny * nz;
  for (int pq = 0; pq < ny * nz; pq++) {
    double s = 0.0;
    for (int k = 0; k < ncomp_k; k++)
      for (int g = 0; g < c->ng; g++)
        for (int a = 0; a < c->na; a++) s += psi[k * ncomp + IDX5(c, g, 0, a, pq / nz, pq % nz)] * c->de[g];
    out[pq] = s * c->du * c->dv;
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
