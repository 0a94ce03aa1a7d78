/* mm_oracle.h -- plain, slow FP64 CPU oracle for the moving-mesh hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library.
 *
 * Layouts are array-of-structs: pos[n][3], W[n][ng] = (rho, rho v, rho e
 * [, rho A]) with ng = 5, or 6 when the entropy column is on (cfg.entropy),
 * grad[n][ng][3] (component-major, then x,y,z).  Faces are either "directed"
 * (every face of every cell, seen from that cell) or "unique" (one record per
 * shared face, i<j, or i==j with a positive image shift).
 */
#ifndef MM_ORACLE_H
#define MM_ORACLE_H
#include <stdint.h>

typedef struct {
    double gamma;      /* ideal-gas adiabatic index, P = (gamma-1) rho eps (Sec. 6)      */
    double cfl;        /* eta_CFL in the per-cell timestep (Sec. 4.2)                     */
    double eta;        /* mesh velocity w = eta v (Sec. 4.2)                              */
    double chi, zeta;  /* roundness correction constants (Sec. 4.2)                       */
    double theta;      /* Duffell-MacFadyen limiter parameter (Sec. 4.1)                  */
    double rho_floor;  /* density floor (Sec. 4.1, value not given in the paper)          */
    double eps_floor;  /* specific internal energy ("temperature") floor (Sec. 4.1)       */
    int limiter;       /* 0 none, 1 S10, 2 S10 then Duffell-MacFadyen, 3 S10 to face centroids */
    int regularize;    /* 1: add the roundness correction to the mesh velocity            */
    int riemann;       /* 0 HLLC, 1 HLL (Sec. 4)                                         */
    int entropy;       /* 1: sixth state column rho A, A = P / rho^gamma, and the switch  */
                       /*    between energy and entropy per cell (Sec. 4.3)               */
    double mach_th;    /* energy equation where the cell's largest shock Mach number is   */
                       /* at least mach_th, entropy equation elsewhere (1.1 in the paper) */
} orc_cfg;

/* States: per cell ng = 5 + entropy values, array of structs (n, ng). */

/* Voronoi tessellation of the periodic box by clipping (Sec. 3).
 * mode 0: brute force over all generators and their 27 images.
 * mode 1: uniform grid of bins, block of bins grown until complete.
 * Directed faces are written for cell 0, then cell 1, ... ; a face is kept
 * when its area exceeds area_rel * (V_box / n)^(2/3).
 * Returns 0 ok, 1 face capacity exceeded, 2 invalid input, 3 internal limit. */
int orc_tessellate(int64_t n, const double *pos, const double *box, int mode, double area_rel,
                   double *volume, double *centroid,
                   int64_t cap, int64_t *nface,
                   int32_t *f_cell, int32_t *f_nb, int32_t *f_shift,
                   double *f_area, double *f_normal, double *f_centroid);

/* Same as orc_tessellate but only for the listed cells (all generators are
 * still candidates); used to time a bounded sample of a large workload. */
int orc_tessellate_subset(int64_t n, const double *pos, const double *box, double area_rel,
                          int64_t m, const int64_t *cells, double *volume, double *centroid,
                          int64_t cap, int64_t *nface, int32_t *f_cell, int32_t *f_nb,
                          int32_t *f_shift, double *f_area, double *f_normal, double *f_centroid);

/* Limited cell-centred gradient of a per-volume field W[n][5] (Sec. 4.1).
 * Unique faces.  grad[n][5][3]. */
void orc_gradient(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const int32_t *fshift,
                  const double *farea, const double *fnormal, const double *fcentroid, const double *centroid,
                  const double *box, const double *W, const orc_cfg *cfg, double *grad);

/* Half-step predictor (Sec. 4.1): Wh = W - dt/2 sum_d A_d(W) dW/dx_d. */
void orc_half_step(int64_t n, const double *W, const double *grad, const orc_cfg *cfg, double dt,
                   double *Wh);

/* Per unique face: reconstruct both sides at the face centroid, floor, boost
 * into the face frame, HLLC, boost back, times area (Sec. 4).  flux[nf][5]. */
void orc_face_flux(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const int32_t *fshift,
                   const double *farea, const double *fnormal, const double *fcentroid,
                   const double *pos, const double *centroid, const double *box,
                   const double *Wh, const double *grad, const double *w, const orc_cfg *cfg,
                   double *flux, double *mach /* [nf] or NULL */, double *vrate /* [nf] or NULL */);

/* Charge update U_i <- U_i - dt sum_j Phi_ij, then cell floors (Sec. 4, 4.1). */
void orc_update(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const double *flux,
                const double *mach /* [nf], used with entropy */, const double *vrate /* [nf], idem */,
                double dt, const double *volume, const orc_cfg *cfg, double *U);

/* Mesh-generator velocity w = eta v (+ roundness correction) (Sec. 4.2). */
void orc_mesh_velocity(int64_t n, const double *pos, const double *U, const double *volume,
                       const double *centroid, const orc_cfg *cfg, double *w);

/* Global CFL timestep min_i eta_CFL R_i / (c_s + |v - w|) (Sec. 4.2). */
double orc_timestep(int64_t n, const double *U, const double *volume, const double *w,
                    const orc_cfg *cfg);

/* Drift r <- r + w dt, wrapped into [0, box). */
void orc_drift(int64_t n, double *pos, const double *w, double dt, const double *box);

/* Pieces exposed for pins. */
void orc_floor_state(const double *W, const orc_cfg *cfg, double *Wout, int *changed);
void orc_euler_flux(const double *W, const double *nrm, double gamma, double *F);
void orc_flux_jacobian(const double *W, int d, double gamma, double *A /* [5][5] */);
/* Lab-frame face flux of two per-volume states across a face with unit
 * normal nrm moving at wface (boost, rotate, HLLC, rotate back, boost back). */
void orc_riemann_lab(const double *WL, const double *WR, const double *nrm, const double *wface,
                     const orc_cfg *cfg, double *F, double *mach /* or NULL */);
/* Contact speed and star pressure of the HLLC model (Davis wave speeds). */
void orc_star_state(const double *primL, const double *primR, double gamma, double *sl, double *ss,
                    double *sr, double *pstar);
/* Largest Mach number of a shock running into either side (0 if none). */
double orc_shock_mach(const double *primL, const double *primR, double gamma);

/* Heun combination (Sec. 6, second-order time integration): U <- (U0 + U)/2
 * for every cell, then the cell floors with the given volumes. */
void orc_heun_average(int64_t n, const double *U0, const double *volume, const orc_cfg *cfg, double *U);
/* One-dimensional HLLC flux in the face frame: prim = (rho, u, v1, v2, P). */
void orc_hllc_1d(const double *primL, const double *primR, double gamma, double *F);
/* One-dimensional HLL flux with the same wave speeds. */
void orc_hll_1d(const double *primL, const double *primR, double gamma, double *F);

#endif
