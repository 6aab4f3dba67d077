/*
 * pbs_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only).
 * See pbs_oracle.c for the method and the readings of the paper it takes.
 */
#ifndef PBS_ORACLE_H
#define PBS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int ny, nz, ng, nu, nv;
  double dy, dz;           /* lateral cell sizes (cm) */
  double u_max, v_max;     /* half-width of the (u,v) box */
  const double *e_faces;   /* ng+1 ascending group faces (MeV) */
} orc_grid;

typedef struct {
  double bk_alpha, bk_p;   /* Bragg-Kleeman range law R = alpha E^p (cm, MeV) */
  double x0;               /* radiation length (g/cm^2) */
  double mp;               /* proton rest energy (MeV) */
  double es;               /* Highland constant (MeV) */
  double sigma_ct;         /* catastrophic removal, mass (cm^2/g) */
  double lambda_p1;        /* exponential energy-transfer rate (1/MeV) */
  double g_alpha, g_beta;  /* Gamma angular-deflection parameters */
  double s_scale;          /* multiplies S (0 switches energy loss off) */
  double ts_scale;         /* multiplies the scattering power */
  int model;               /* 0: Bragg-Kleeman + Highland; 1: the paper's Appendix A
                              (Bethe-Bloch with Bragg additivity, screened Rutherford) */
  double t_scale;          /* multiplies the straggling coefficient of Appendix A.2 (0: none) */
} orc_phys;

typedef struct {
  double e0, sigma_e, y0, z0, sigma_y, sigma_z, u0, v0, sigma_u, sigma_v;
} orc_beam;

typedef struct {
  int n_scatter;           /* K: components psi_p, psi_s1..psi_sK */
  int scheme;              /* 0 Strang + CN, 1 first-order splitting */
  int do_energy, do_transport, do_angular;
} orc_march_opts;

typedef struct orc_ctx orc_ctx;

orc_ctx *orc_create(const orc_grid *g, const orc_phys *ph);
void orc_destroy(orc_ctx *c);
void orc_get_tables(const orc_ctx *c, double *s_face, double *ts, double *sig, double *p1, double *p2,
                    double *u, double *v);
double orc_highland(const orc_phys *ph, double e);
double orc_bethe_water(const orc_phys *ph, double e);
double orc_bethe_element(const orc_phys *ph, double z, double a, double e);
double orc_sigma_tr_element(const orc_phys *ph, double z, double a, double e);
double orc_scat_power_water(const orc_phys *ph, double e);
double orc_williams_water(const orc_phys *ph, double e);
void orc_set_sigma(orc_ctx *c, const double *sig);
void orc_set_straggling_table(orc_ctx *c, const double *t_face);
void orc_set_straggling_cn(orc_ctx *c, int full);
void orc_get_straggling(const orc_ctx *c, double *t_face, double *s_base);
void orc_straggle_blocks(const orc_ctx *c, int g, double rho, double alo[2][2], double agg[2][2],
                         double aup[2][2]);
void orc_straggle_apply(const orc_ctx *c, double rho, const double *x, double *out);
void orc_energy_blocks(const orc_ctx *c, int g, double rho, double agg[2][2], double aup[2][2]);
void orc_energy_apply(const orc_ctx *c, double rho, const double *x, double *out);
double orc_energy_cn_lane(const orc_ctx *c, double rho, double h, double *x, const double *src_sum,
                          double *edep_w);
void orc_energy_substep(const orc_ctx *c, double h, const double *rho_yz, double *psi, const double *src_sum,
                        double *edep_yz, double *edep_w_yz);
void orc_source(const orc_ctx *c, const double *rho_yz, const double *prev, double *out);
void orc_transport_substep(const orc_ctx *c, double h, double *psi);
void orc_transport_apply(const orc_ctx *c, double uu, double vv, const double *f, double *out, int first_order);
void orc_set_transport_cn(orc_ctx *c, int cn);
void orc_angular_substep(const orc_ctx *c, double h, const double *rho_yz, double *psi);
void orc_set_angular_exact(orc_ctx *c, int exact);
void orc_init_beam(const orc_ctx *c, const orc_beam *b, double *psi);
int orc_march(const orc_ctx *c, const orc_march_opts *o, const orc_beam *b, const double *rho, int n_steps,
              double dx, double *psi, double *dose, double *edep_w, double *fluence);
void orc_fluence(const orc_ctx *c, const double *psi, int ncomp_k, double *out);
int orc_num_threads(void);
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
