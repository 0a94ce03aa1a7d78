// mm_internal.cuh -- shared declarations of the CUDA moving-mesh library.
//
// Every mesh is a set of B independent periodic boxes stored back to back
// (a single box is B = 1): cell c belongs to box cbox[c]; box b has its own
// grid of bins (a contiguous range of the global bin array), size, face-area
// threshold and timestep dt[b].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mm.h"

namespace mm {

// Per-cell fixed capacities of the clipping kernel (Sec. 3).  A cell that
// exceeds one is clipped again by the large instance of the same kernel
// (twice the planes, vertices and faces, 128 search rings), whose faces
// go to an overflow row of its own; only a cell that exceeds those too
// reports MM_ECAPACITY.
constexpr int PMAX = 64;    // planes that ever cut the cell (6 box planes included)
constexpr int TMAX = 128;   // vertices (triangles of the dual) alive at once
constexpr int NSTAGE = 32;  // vertices created by one cut
constexpr int MAXF = 48;    // faces written per cell
constexpr int MAXRING = 48; // search rings before giving up
constexpr int PMAX_BIG = 128, TMAX_BIG = 256, NSTAGE_BIG = 64, MAXF_BIG = 128, MAXRING_BIG = 128;
constexpr int CLIP_MAX_WARPS = 8;  // warps (cells) per block of the clipper, tunable at run time
// Overflow rows reserved when the count of retried cells is not known in
// advance (graph mode); mm_tessellate sizes them to the count it reads.
constexpr int RETRY_ROWS_FIXED = 256;

// Device status word, read by the host after a tessellation.
enum : int {
    ST_EINVAL = 1,
    ST_ECAP_CAND = 2,
    ST_ECAP_PLANE = 4,
    ST_ECAP_TRI = 8,
    ST_ECAP_STAGE = 16,
    ST_ECAP_FACE = 32,
    ST_ECAP_RING = 64,
    ST_EDEGEN = 128,     // two generators at one position
    ST_ECAP_MESH = 256,  // more unique faces or incidences than a fixed capacity (graph mode)
    ST_ECAP_RETRY = 512, // more retried cells than overflow rows (graph mode)
    ST_EDEGEN_CUT = 1024, // a cut whose removed vertices are not a cap (near-degenerate generators)
};
// Flags that send a cell to the large clipper instead of failing: its
// capacities, and an inconsistent cut, which the large clipper retries with
// the strict tie rule (the retry entry is then ~w instead of w).
constexpr int ST_RETRYABLE =
    ST_ECAP_CAND | ST_ECAP_PLANE | ST_ECAP_TRI | ST_ECAP_STAGE | ST_ECAP_FACE | ST_ECAP_RING | ST_EDEGEN_CUT;

struct DevStatus {
    int flags;
    int bad_cell;
    int max_cand, max_planes, max_tris;
    int multi_ring;
    unsigned long long cuts;
    unsigned long long pred64;   // FP64 plane tests  (q.v > o: 5 flops)
    unsigned long long solve64;  // FP64 three-plane solves (51 flops)
    unsigned long long fan64;    // FP64 fan terms of the face geometry
    unsigned long long tested;   // candidates tested against the cell
    int nretry;                  // cells sent to the large clipper
};

// One periodic box of a batch.
struct BoxDev {
    int g[3];      // bins per axis
    int bin_off;   // first bin of this box in the global bin array
    double bs[3];  // bin edge per axis
    double ibs[3]; // 1 / bin edge (bin of x: floor(x * ibs))
    double L[3];   // box size
    double amin;   // faces with area <= amin are dropped
    float Lf[3], bsf[3], ibsf[3];  // FP32 roundings of L, bs, ibs (the clipper's setup arithmetic)
};

struct Slots {         // per-cell face slots written by the clipper
    int *cnt;          // [n]: faces in the cell's row; -(k+1): they are in overflow row k
    int *nb;           // [n*MAXF]
    unsigned char *sh; // [n*MAXF] shift code
    double *area;      // [n*MAXF]
    double *fc;        // [3][n*MAXF] face centroid relative to the generator
    // overflow rows of the cells retried by the large clipper, MAXF_BIG slots each
    int64_t orows;      // rows reserved
    int *ocnt;          // [orows] faces in the row
    int *onb;           // [orows*MAXF_BIG]
    unsigned char *osh; // [orows*MAXF_BIG]
    double *oarea;      // [orows*MAXF_BIG]
    double *ofc;        // [3][orows*MAXF_BIG]
    int *retry;         // [n] binned indices w of the retried cells (~w: retry with the strict tie rule)
};

// Face confirmation state of the overflow rows: two mask words and a partner
// slot per overflow slot (the main rows use the per-cell masks and partners).
struct OvfFaces {
    unsigned long long *emit, *conf;  // [2*orows]
    signed char *partner;             // [orows*MAXF_BIG]
    const int *nretry;                // cells re-clipped (0: no overflow row is in use)
};

// kernels' host launchers (stream-ordered, no syncs)
void launch_fill_cbox(const long long *box_off, int nbox, int64_t n, int *cbox, cudaStream_t s);
void launch_bin_count(const double *pos, int64_t n, const BoxDev *boxes, const int *cbox, int *bin_of, int *count,
                      DevStatus *st, cudaStream_t s);
void launch_bin_scatter(const double *pos, int64_t n, const int *bin_of, const int *start, int *cursor,
                        double4_32a *sorted, cudaStream_t s);
void launch_bin_sort(const int *start, int64_t nbins, double4_32a *sorted, float4 *sortedf, cudaStream_t s);
// exclusive scan of in[0..n) into out[0..n], out[n] = total; tmp >= scan_tmp_size(n) ints
size_t scan_tmp_size(int64_t n);
void launch_scan(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s);

// vol receives each cell's volume and cen its first moment about the
// generator ([3][n]); launch_face_write turns the moment into the centroid.
// The main clipper (every cell, fixed capacities; a cell over a capacity is
// appended to sl.retry) and the large clipper (the cells of sl.retry, their
// faces to the overflow rows; a launch of sl.orows warps handles the first
// min(nretry, orows) of them and flags the rest).
void launch_clip(const double4_32a *sorted, const float4 *sortedf, const int *start, int64_t n, const BoxDev *boxes,
                 const int *cbox,
                 int precision, int collect, int warps, int cand_cap, int sort, double *vol, double *cen,
                 Slots sl, DevStatus *st, cudaStream_t s);
void launch_clip_big(const double4_32a *sorted, const float4 *sortedf, const int *start, int64_t n,
                     const BoxDev *boxes, const int *cbox, int precision, int collect, int cand_cap, double *vol,
                     double *cen, Slots sl, DevStatus *st, cudaStream_t s);

// (also reports ST_EDEGEN_CUT for a face far above the area threshold that
// the neighbour does not have)
void launch_face_confirm(int64_t n, Slots sl, OvfFaces ov, const BoxDev *boxes, const int *cbox, DevStatus *st,
                         unsigned long long *emit_mask, unsigned long long *conf_mask, signed char *partner,
                         int *emit_cnt, int *conf_cnt, cudaStream_t s);
void launch_face_write(int64_t n, const double *pos, const BoxDev *boxes, const int *cbox, Slots sl, OvfFaces ov,
                       const unsigned long long *emit_mask, const unsigned long long *conf_mask,
                       const signed char *partner, const int *face_off, const int *inc_off,
                       int *face_i, int *face_j, int *face_shift, double *face_area, double *face_normal,
                       double *face_cen, int64_t fcap, int *inc_face, int64_t icap, const double *vol,
                       double *cen, DevStatus *st, cudaStream_t s);

struct MeshDev {
    int64_t n;           // cells
    int64_t nf;          // unique faces (host value; see nf_dev)
    int64_t fs;          // face capacity: row stride of the [3][.] face arrays and of the flux rows
    const int *nf_dev;   // if set, the face count is read from here on the device (graph mode)
    const int *cbox;     // [n] box of each cell
    const double *boxL;  // [B][3] box sizes
    const int *face_i, *face_j, *face_shift;
    const double *area, *normal, *fcen;
    const double *vol, *cen;
    const int *inc_off, *inc_face;
    // Order in which the kernels that loop over a cell's incident faces take
    // the cells: within every aligned run of CELL_ORDER_BLOCK entries, that
    // run's cells by their number of incident faces (then by index), so the
    // lanes of a warp run loops of nearly equal length.  NULL: index order.
    const int *order;
};
constexpr int CELL_ORDER_BLOCK = 128;

// The cell a thread of an incident-face kernel takes (t < n).
__device__ __forceinline__ int64_t cell_of(const MeshDev &m, int64_t t) { return m.order ? m.order[t] : t; }
void launch_cell_order(int64_t n, const int *inc_off, int *order, cudaStream_t s);

struct HydroCfg {
    double gamma, cfl, eta, chi, zeta, theta, rho_floor, eps_floor;
    double mach_th;  // energy/entropy switch threshold (Sec. 4.3)
    double igm1;     // 1 / (gamma - 1), formed once on the host
    double kmach;    // (gamma + 1) / (2 gamma), the shock Mach relation's factor
    double rhoa_floor;  // rho A of the floor state: rho_f (gamma-1) rho_f eps_f / rho_f^gamma
    int limiter, regularize, riemann;
    int entropy;     // 1: a sixth state column rho A and the switch
};

// FP32 records of the mixed-precision hydro path (see mm_hydro32.cu).
struct Mixed {
    int2 *fij;     // [F]
    float4 *fa;    // [F]   area, normal
    float4 *fq;    // [F]   r_j' - r_i, (x_f - r_i).x
    float2 *ff;    // [F]   (x_f - r_i).y, .z
    float4 *cw;    // [2n]  W^n, c - r
    float4 *ch;    // [2n]  W^(n+1/2), c - r
    float4 *grad;  // [4n]  limited gradient of W^(n+1/2)
    float4 *wv;    // [n]   mesh velocity
    float4 *flux;  // [2F]  A F
};

// dt arguments are per-box arrays [B] indexed through cbox.  Launchers over
// faces size their grid by the face capacity when the count lives on the
// device (graph mode).
void launch_mixed_step(const MeshDev &m, const HydroCfg &c, const double *pos, const double *w, const double *dt,
                       Mixed x, double *U, cudaStream_t s, void (*mark)(void *, int, bool), void *mark_arg);
// geo [6][fs] doubles: A n and d per face (launch_face_geom), followed by
// [3][fs] floats: d rounded to FP32.  With W_half the
// half-step predictor runs and M^-1 is stored in minv [9][n]; otherwise the
// limited gradient goes to grad, with M^-1 read from minv when minv_in.
void launch_face_geom(const MeshDev &m, double *geo, cudaStream_t s);
void launch_gradient(const MeshDev &m, const HydroCfg &c, const double *W, const double *geo, double *minv,
                     bool minv_in, double *grad, double *W_half, const double *dt, cudaStream_t s);
void launch_face_flux(const MeshDev &m, const HydroCfg &c, const double *pos, const double *w,
                      const double *Wh, const double *grad, double *flux, cudaStream_t s);
void launch_states(const MeshDev &m, const HydroCfg &c, const double *U, double *W, cudaStream_t s);
void launch_heun_average(const MeshDev &m, const HydroCfg &c, const double *U0, double *U, cudaStream_t s);
void launch_update(const MeshDev &m, const HydroCfg &c, const double *flux, const double *dt, double *U,
                   cudaStream_t s);
void launch_mesh_velocity(const MeshDev &m, const HydroCfg &c, const double *pos, const double *U,
                          double *w, double *dt_min, cudaStream_t s);
void launch_dt_init(double *dt, int nbox, cudaStream_t s);
void launch_timestep(const MeshDev &m, const HydroCfg &c, const double *U, const double *w, double *dt_min,
                     cudaStream_t s);
void launch_drift(double *pos, int64_t n, const double *w, const double *dt, const int *cbox, const double *boxL,
                  cudaStream_t s);
void launch_prims_to_charges(const MeshDev &m, const HydroCfg &c, const double *rho, const double *vel,
                             const double *P, double *U, cudaStream_t s);
void launch_totals(const double *U, int64_t n, double *partial, int nblocks, double *totals, cudaStream_t s);

// The face count a kernel over faces must honour.
__device__ __forceinline__ int64_t face_count(const MeshDev &m) { return m.nf_dev ? (int64_t)*m.nf_dev : m.nf; }

// Grid size of a launch over faces.
inline int64_t face_launch_count(const MeshDev &m) { return m.nf_dev ? m.fs : m.nf; }

}  // namespace mm
