// mm_hydro.cu -- the finite-volume stages of one step on the Voronoi mesh
// (Sec. 4, 4.1, 4.2).  All loops are cell-centric over the incident-face
// lists (gradients, update) or face-centric over unique faces (fluxes); no
// atomics touch the conserved data, so results are bitwise reproducible.
#include "mm_internal.cuh"
#include "mm_riemann.cuh"

namespace mm {

constexpr unsigned FULL_MASK_HYDRO = 0xffffffffu;

#ifndef MM_GRAD_MINBLOCKS
#define MM_GRAD_MINBLOCKS 1  // resident blocks per SM the gradient kernel is compiled for
#endif

// Flip the sign of x when the mask has the sign bit set (an integer op).
__device__ __forceinline__ double flip(double x, long long smask)
{
    return __longlong_as_double(__double_as_longlong(x) ^ smask);
}

// One axis of an image offset: digit 0, 1, 2 of the image code means -L, 0, +L.
__device__ __forceinline__ double image_axis(int digit, double L)
{
    return digit == 1 ? 0.0 : (digit == 2 ? L : -L);
}

template <int NG>
__device__ __forceinline__ void loadw(const double *S, int64_t n, int64_t i, double inv_v, double w[NG])
{
#pragma unroll
    for (int k = 0; k < NG; ++k) w[k] = S[k * n + i] * inv_v;
}
__device__ __forceinline__ void load5(const double *S, int64_t n, int64_t i, double inv_v, double w[5])
{
    loadw<5>(S, n, i, inv_v, w);
}

__device__ __forceinline__ bool apply_floor(double W[5], double rho_floor, double eps_floor)
{
    return apply_floor_t<double>(W, rho_floor, eps_floor);
}

// ---------------------------------------------------------------------------
// Face geometry of the gradient (Sec. 4.1), once per mesh and step: per
// unique face the area-weighted normal A n and the centroid separation
// d = c_j + s L - c_i, both seen from side i (side j sees -A n, -d).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_face_geom(MeshDev m, double *__restrict__ geo)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= face_count(m)) return;
    const int64_t n = m.n, fs = m.fs;
    const int i = m.face_i[f], j = m.face_j[f];
    const int code = m.face_shift[f];
    const double *L = m.boxL + 3 * m.cbox[i];
    const double A = m.area[f];
    geo[f] = A * m.normal[f];
    geo[fs + f] = A * m.normal[fs + f];
    geo[2 * fs + f] = A * m.normal[2 * fs + f];
    const double dx = m.cen[j] + image_axis(code % 3, L[0]) - m.cen[i];
    const double dy = m.cen[n + j] + image_axis((code / 3) % 3, L[1]) - m.cen[n + i];
    const double dz = m.cen[2 * n + j] + image_axis(code / 9, L[2]) - m.cen[2 * n + i];
    geo[3 * fs + f] = dx;
    geo[4 * fs + f] = dy;
    geo[5 * fs + f] = dz;
    // FP32 roundings of d after the six FP64 rows, for the limiter's screening
    float *g32 = reinterpret_cast<float *>(geo + 6 * fs);
    g32[f] = (float)dx;
    g32[fs + f] = (float)dy;
    g32[2 * fs + f] = (float)dz;
}

void launch_face_geom(const MeshDev &m, double *geo, cudaStream_t s)
{
    const int64_t nfl = face_launch_count(m);
    if (nfl == 0) return;
    k_face_geom<<<(int)((nfl + 255) / 256), 256, 0, s>>>(m, geo);
}

// The running minima and maxima of the limiter are kept as order-preserving
// integers (okey): integer comparisons in place of FP64 min/max.
__device__ __forceinline__ long long kmax(long long a, long long b) { return a > b ? a : b; }
// Delta = g . d with explicitly rounded operations, so the screened and the
// exhaustive limiter paths form the same bits
__device__ __forceinline__ double deldot(double g0, double g1, double g2, double dx, double dy, double dz)
{
    return __fma_rn(g2, dz, __fma_rn(g1, dy, __dmul_rn(g0, dx)));
}
__device__ __forceinline__ long long kmin(long long a, long long b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// Gradient + limiter (+ half-step predictor when PREDICT)
// ---------------------------------------------------------------------------
// NG = 5 state columns, or 6 with the entropy column rho A (Sec. 4.3), which
// is treated like the others and advected in the predictor.  The geometric
// matrix M depends on the mesh only: the predictor pass stores M^-1 per cell
// ([9][n], row major) and the second pass on the same mesh (MINV_IN) reads it.
template <bool PREDICT, bool MINV_IN, int NG>
__global__ void __launch_bounds__(128, MM_GRAD_MINBLOCKS) k_gradient(MeshDev m, HydroCfg c, const double *__restrict__ S,
                                                  const double *__restrict__ geo, double *__restrict__ minv,
                                                  double *__restrict__ grad, double *__restrict__ Wh,
                                                  const double *__restrict__ dtp)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n, fs = m.fs;
    if (t >= n) return;
    const int64_t i = cell_of(m, t);
    double Wi[NG];
    loadw<NG>(S, n, i, 1.0, Wi);
    const int e0 = m.inc_off[i], e1 = m.inc_off[i + 1];

    // M = 1/2 sum A n (x) d,  b_k = 1/2 sum A (W_o - W_i)_k n; the signs of
    // A n and d flip together on side j, so M takes the stored vectors as
    // they are and b takes the sign on W_o - W_i.  (Both are summed without
    // the factor 1/2, which cancels exactly in M^-1 b.)
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double b[3 * NG];
    long long kx[NG], kn[NG];  // running max / min of W over the cell and its neighbours
#pragma unroll
    for (int k = 0; k < NG; ++k) { kx[k] = okey(Wi[k]); kn[k] = kx[k]; }
#pragma unroll
    for (int k = 0; k < 3 * NG; ++k) b[k] = 0.0;
    for (int e = e0; e < e1; ++e) {
        int f = m.inc_face[e];
        const bool fwd = f >= 0;
        if (!fwd) f = ~f;
        const int o = fwd ? m.face_j[f] : m.face_i[f];
        const long long sm = fwd ? 0LL : (long long)0x8000000000000000ULL;
        const double ax = geo[f], ay = geo[fs + f], az = geo[2 * fs + f];
        if (!MINV_IN) {
            const double dx = geo[3 * fs + f], dy = geo[4 * fs + f], dz = geo[5 * fs + f];
            M[0] += ax * dx; M[1] += ax * dy; M[2] += ax * dz;
            M[3] += ay * dx; M[4] += ay * dy; M[5] += ay * dz;
            M[6] += az * dx; M[7] += az * dy; M[8] += az * dz;
        }
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const double wo = S[k * n + o];
            const double dw = flip(wo - Wi[k], sm);
            b[3 * k + 0] += ax * dw;
            b[3 * k + 1] += ay * dw;
            b[3 * k + 2] += az * dw;
            const long long kw = okey(wo);
            kx[k] = kmax(kx[k], kw);
            kn[k] = kmin(kn[k], kw);
        }
    }
    double mi[9];
    if (MINV_IN) {
#pragma unroll
        for (int r = 0; r < 9; ++r) mi[r] = minv[r * n + i];
    } else {
        // M^-1 by the adjugate
        const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
        const double c10 = M[2] * M[7] - M[1] * M[8], c11 = M[0] * M[8] - M[2] * M[6], c12 = M[1] * M[6] - M[0] * M[7];
        const double c20 = M[1] * M[5] - M[2] * M[4], c21 = M[2] * M[3] - M[0] * M[5], c22 = M[0] * M[4] - M[1] * M[3];
        const double idet = 1.0 / (M[0] * c00 + M[1] * c01 + M[2] * c02);
        mi[0] = c00 * idet; mi[1] = c10 * idet; mi[2] = c20 * idet;
        mi[3] = c01 * idet; mi[4] = c11 * idet; mi[5] = c21 * idet;
        mi[6] = c02 * idet; mi[7] = c12 * idet; mi[8] = c22 * idet;
        if (PREDICT) {
#pragma unroll
            for (int r = 0; r < 9; ++r) minv[r * n + i] = mi[r];
        }
    }
    double g[3 * NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
        const double b0 = b[3 * k], b1 = b[3 * k + 1], b2 = b[3 * k + 2];
        g[3 * k + 0] = mi[0] * b0 + mi[1] * b1 + mi[2] * b2;
        g[3 * k + 1] = mi[3] * b0 + mi[4] * b1 + mi[5] * b2;
        g[3 * k + 2] = mi[6] * b0 + mi[7] * b1 + mi[8] * b2;
    }
    if (c.limiter >= 1) {
        // S10: alpha = min(1, min_j psi_ij); with c_max = W_max - W_i >= 0 and
        // c_min = W_min - W_i <= 0 the minimum over j is attained at the
        // largest positive and the most negative Delta_ij = g . d_ij.
        long long kdx[NG], kdn[NG];  // max / min of Delta, starting from 0
#pragma unroll
        for (int k = 0; k < NG; ++k) { kdx[k] = 0; kdn[k] = 0; }
        bool exhaustive = c.limiter != 1;
        if (c.limiter == 1) {
            // S10 with centroid separations: Delta in FP32 from FP32 copies of
            // g and d, whose error is below B = 8e-7 |g|_1 max_j |d_j|_1 (five
            // roundings of 2^-24 plus margin).  Where the largest Delta leads
            // the runner-up by more than 2B (the value 0 competing too), the
            // FP32 leader is the exact maximum and only its Delta is formed in
            // FP64; likewise for the minimum.  Otherwise (ties, lattices) the
            // exhaustive FP64 pass below decides.  The result is the same bits.
            const float *g32 = reinterpret_cast<const float *>(geo + 6 * fs);
            float gf[3 * NG];
#pragma unroll
            for (int k = 0; k < 3 * NG; ++k) gf[k] = (float)g[k];
            float m1[NG], m2[NG], n1[NG], n2[NG];
            int i1[NG], j1[NG];
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                m1[k] = 0.0f; n1[k] = 0.0f; i1[k] = -1; j1[k] = -1;
                m2[k] = -__int_as_float(0x7f800000); n2[k] = __int_as_float(0x7f800000);
            }
            float dl1 = 0.0f;
            for (int e = e0; e < e1; ++e) {
                int f = m.inc_face[e];
                const unsigned sm = f >= 0 ? 0u : 0x80000000u;
                if (f < 0) f = ~f;
                const float dx = __uint_as_float(__float_as_uint(g32[f]) ^ sm);
                const float dy = __uint_as_float(__float_as_uint(g32[fs + f]) ^ sm);
                const float dz = __uint_as_float(__float_as_uint(g32[2 * fs + f]) ^ sm);
                dl1 = fmaxf(dl1, fabsf(dx) + fabsf(dy) + fabsf(dz));
#pragma unroll
                for (int k = 0; k < NG; ++k) {
                    const float del = fmaf(gf[3 * k], dx, fmaf(gf[3 * k + 1], dy, gf[3 * k + 2] * dz));
                    if (del > m1[k]) { m2[k] = m1[k]; m1[k] = del; i1[k] = e; } else m2[k] = fmaxf(m2[k], del);
                    if (del < n1[k]) { n2[k] = n1[k]; n1[k] = del; j1[k] = e; } else n2[k] = fminf(n2[k], del);
                }
            }
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                const float b2 = 2.0f * (8e-7f * (fabsf(gf[3 * k]) + fabsf(gf[3 * k + 1]) + fabsf(gf[3 * k + 2])) * dl1 + 1e-36f);
                // a zero gradient (a uniform column) stays zero whatever its extremes: no tie to settle
                const bool gzero = ((__double_as_longlong(g[3 * k]) | __double_as_longlong(g[3 * k + 1]) |
                                     __double_as_longlong(g[3 * k + 2])) << 1) == 0;
                if (!gzero && (!(m1[k] - m2[k] > b2) || !(n2[k] - n1[k] > b2))) exhaustive = true;
                if (i1[k] >= 0) {
                    int f = m.inc_face[i1[k]];
                    const long long sm = f >= 0 ? 0LL : (long long)0x8000000000000000ULL;
                    if (f < 0) f = ~f;
                    kdx[k] = okey(deldot(g[3 * k], g[3 * k + 1], g[3 * k + 2], flip(geo[3 * fs + f], sm),
                                         flip(geo[4 * fs + f], sm), flip(geo[5 * fs + f], sm)));
                }
                if (j1[k] >= 0) {
                    int f = m.inc_face[j1[k]];
                    const long long sm = f >= 0 ? 0LL : (long long)0x8000000000000000ULL;
                    if (f < 0) f = ~f;
                    kdn[k] = okey(deldot(g[3 * k], g[3 * k + 1], g[3 * k + 2], flip(geo[3 * fs + f], sm),
                                         flip(geo[4 * fs + f], sm), flip(geo[5 * fs + f], sm)));
                }
            }
        }
        const double cix = m.cen[i], ciy = m.cen[n + i], ciz = m.cen[2 * n + i];
        const double *L = m.boxL + 3 * m.cbox[i];
        if (exhaustive) {
#pragma unroll
        for (int k = 0; k < NG; ++k) { kdx[k] = 0; kdn[k] = 0; }
        for (int e = e0; e < e1; ++e) {
            int f = m.inc_face[e];
            const bool fwd = f >= 0;
            if (!fwd) f = ~f;
            double dx, dy, dz;
            if (c.limiter == 3) {
                // to the face centroid, in this cell's frame (subtract the image offset on the j side)
                const int code = m.face_shift[f];
                const double sh = fwd ? 0.0 : 1.0;
                dx = m.fcen[f] - sh * image_axis(code % 3, L[0]) - cix;
                dy = m.fcen[fs + f] - sh * image_axis((code / 3) % 3, L[1]) - ciy;
                dz = m.fcen[2 * fs + f] - sh * image_axis(code / 9, L[2]) - ciz;
            } else {
                const long long sm = fwd ? 0LL : (long long)0x8000000000000000ULL;
                dx = flip(geo[3 * fs + f], sm);
                dy = flip(geo[4 * fs + f], sm);
                dz = flip(geo[5 * fs + f], sm);
            }
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                const double del = deldot(g[3 * k], g[3 * k + 1], g[3 * k + 2], dx, dy, dz);
                const long long kd = okey(del);
                kdx[k] = kmax(kdx[k], kd);
                kdn[k] = kmin(kdn[k], kd);
            }
        }
        }
        double al[NG];
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            // the ratios matter only below 1 (min(1, x)), so most cells skip the
            // FP64 divisions: x < 1 exactly when the numerator is the smaller
            double a = 1.0;
            const double up = okey_value(kx[k]) - Wi[k], dn = okey_value(kn[k]) - Wi[k];
            const double dmax = okey_value(kdx[k]), dmin = okey_value(kdn[k]);
            if (kdx[k] > 0 && up < dmax) a = fmin(a, up / dmax);
            if (kdn[k] < 0 && dn > dmin) a = fmin(a, dn / dmin);
            al[k] = a;
        }
        if (c.limiter == 2) {
            // DM: min_j max(0, theta (W_j - W_i) / Delta_ij) with the unlimited
            // gradient, tracked as a fraction (num, den > 0) to avoid a division
            // per face.  A neighbour counts only where Delta is nonzero beyond
            // the rounding of g and d, 2^-40 |g|_1 |d|_1: toward the equal-valued
            // transverse neighbours of a lattice Delta is zero in exact
            // arithmetic.  A pass of its own, after the S10 extremes are dead.
            double rn[NG], rd[NG], gl[NG];
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                rn[k] = 1.0; rd[k] = 1.0;
                gl[k] = 0x1p-40 * (fabs(g[3 * k]) + fabs(g[3 * k + 1]) + fabs(g[3 * k + 2]));
            }
            for (int e = e0; e < e1; ++e) {
                int f = m.inc_face[e];
                const bool fwd = f >= 0;
                if (!fwd) f = ~f;
                const long long sm = fwd ? 0LL : (long long)0x8000000000000000ULL;
                const double dx = flip(geo[3 * fs + f], sm), dy = flip(geo[4 * fs + f], sm),
                             dz = flip(geo[5 * fs + f], sm);
                const double dl = fabs(dx) + fabs(dy) + fabs(dz);
                const int o = fwd ? m.face_j[f] : m.face_i[f];
#pragma unroll
                for (int k = 0; k < NG; ++k) {
                    const double del = deldot(g[3 * k], g[3 * k + 1], g[3 * k + 2], dx, dy, dz);
                    if (!(fabs(del) > gl[k] * dl)) continue;
                    double num = c.theta * (S[k * n + o] - Wi[k]);
                    double den = del;
                    if (den < 0.0) { num = -num; den = -den; }
                    if (num < 0.0) num = 0.0;
                    if (num * rd[k] < rn[k] * den) { rn[k] = num; rd[k] = den; }
                }
            }
#pragma unroll
            for (int k = 0; k < NG; ++k) al[k] *= fmin(1.0, rn[k] / rd[k]);
        }
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            g[3 * k] *= al[k];
            g[3 * k + 1] *= al[k];
            g[3 * k + 2] *= al[k];
        }
    }
    if (!PREDICT) {
#pragma unroll
        for (int k = 0; k < 3 * NG; ++k) grad[k * n + i] = g[k];
        return;
    }
    // half-step predictor: dW/dt = -div F written through the chain rule on
    // (rho, m, E):  d_d u_k = (d_d m_k - u_k d_d rho) / rho,
    // d_d P = (gamma-1)(d_d E - u . d_d m + |u|^2/2 d_d rho)
    const double gm1 = c.gamma - 1.0;
    const double ir = 1.0 / Wi[0];
    const double ux = Wi[1] * ir, uy = Wi[2] * ir, uz = Wi[3] * ir;
    const double u2 = ux * ux + uy * uy + uz * uz;
    const double P = gm1 * (Wi[4] - 0.5 * Wi[0] * u2);
    const double u[3] = {ux, uy, uz};
    double du[3][3];  // du[k][d] = d u_k / d x_d
    double dP[3];
    double divu = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double drho = g[d];
#pragma unroll
        for (int k = 0; k < 3; ++k) du[k][d] = (g[3 * (1 + k) + d] - u[k] * drho) * ir;
        dP[d] = gm1 * (g[12 + d] - (ux * g[3 + d] + uy * g[6 + d] + uz * g[9 + d]) + 0.5 * u2 * drho);
        divu += du[d][d];
    }
    double rate[5];
    rate[0] = -(g[3] + g[7] + g[11]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) s += u[d] * g[3 * (1 + k) + d];
        rate[1 + k] = -(s + Wi[1 + k] * divu) - dP[k];
    }
    {
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) s += u[d] * (g[12 + d] + dP[d]);
        rate[4] = -(s + (Wi[4] + P) * divu);
    }
    const double hdt = 0.5 * dtp[m.cbox[i]];
#pragma unroll
    for (int k = 0; k < 5; ++k) Wh[k * n + i] = Wi[k] + hdt * rate[k];
    if constexpr (NG == 6) {
        // d_t (rho A) = -(u . grad(rho A) + rho A div u)
        const double r5 = -(ux * g[15] + uy * g[16] + uz * g[17] + Wi[5] * divu);
        Wh[5 * n + i] = Wi[5] + hdt * r5;
    }
}

template <int NG>
static void launch_gradient_t(const MeshDev &m, const HydroCfg &c, const double *W, const double *geo, double *minv,
                              bool minv_in, double *grad, double *W_half, const double *dt, cudaStream_t s)
{
    const int nb = (int)((m.n + 127) / 128);
    if (W_half) k_gradient<true, false, NG><<<nb, 128, 0, s>>>(m, c, W, geo, minv, grad, W_half, dt);
    else if (minv_in) k_gradient<false, true, NG><<<nb, 128, 0, s>>>(m, c, W, geo, minv, grad, W_half, dt);
    else k_gradient<false, false, NG><<<nb, 128, 0, s>>>(m, c, W, geo, minv, grad, W_half, dt);
}

void launch_gradient(const MeshDev &m, const HydroCfg &c, const double *W, const double *geo, double *minv,
                     bool minv_in, double *grad, double *W_half, const double *dt, cudaStream_t s)
{
    if (c.entropy) launch_gradient_t<6>(m, c, W, geo, minv, minv_in, grad, W_half, dt, s);
    else launch_gradient_t<5>(m, c, W, geo, minv, minv_in, grad, W_half, dt, s);
}

// ---------------------------------------------------------------------------
// Face fluxes: reconstruct, floor, boost into the face frame, HLLC, boost back
// ---------------------------------------------------------------------------
using FaceState = FaceStateT<double>;

// With NG = 6 the flux rows 5, 6 and 7 hold the entropy flux A F_(rho A), the
// face's shock Mach number and its swept-volume rate A (w_f . n).
template <int NG>
__global__ void __launch_bounds__(128) k_face_flux(MeshDev m, HydroCfg c, const double *__restrict__ pos,
                                                   const double *__restrict__ w, const double *__restrict__ Wh,
                                                   const double *__restrict__ grad, double *__restrict__ flux)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= face_count(m)) return;
    const int64_t n = m.n, fs = m.fs;
    const int i = m.face_i[f], j = m.face_j[f];
    const int code = m.face_shift[f];
    const double *Lb = m.boxL + 3 * m.cbox[i];
    const double ox = image_axis(code % 3, Lb[0]), oy = image_axis((code / 3) % 3, Lb[1]),
                 oz = image_axis(code / 9, Lb[2]);
    const double fx = m.fcen[f], fy = m.fcen[fs + f], fz = m.fcen[2 * fs + f];
    const double nx = m.normal[f], ny = m.normal[fs + f], nz = m.normal[2 * fs + f];
    // reconstruction to the face centroid: W_face = W_half + (x_f - c) . grad
    const double dlx = fx - m.cen[i], dly = fy - m.cen[n + i], dlz = fz - m.cen[2 * n + i];
    const double drx = fx - (m.cen[j] + ox), dry = fy - (m.cen[n + j] + oy), drz = fz - (m.cen[2 * n + j] + oz);
    double WL[NG], WR[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
        WL[k] = Wh[k * n + i] + dlx * grad[(3 * k) * n + i] + dly * grad[(3 * k + 1) * n + i] + dlz * grad[(3 * k + 2) * n + i];
        WR[k] = Wh[k * n + j] + drx * grad[(3 * k) * n + j] + dry * grad[(3 * k + 1) * n + j] + drz * grad[(3 * k + 2) * n + j];
    }
    const bool vac_l = !(WL[0] >= c.rho_floor), vac_r = !(WR[0] >= c.rho_floor);
    double irl, irr, kel, ker;
    apply_floor_ir_t<double>(WL, c.rho_floor, c.eps_floor, irl, kel);
    apply_floor_ir_t<double>(WR, c.rho_floor, c.eps_floor, irr, ker);
    if constexpr (NG == 6) {
        // rho A at the face: a state reset to the density floor takes the
        // floor state's own A; otherwise the reconstruction, not below 0
        WL[5] = vac_l ? c.rhoa_floor : fmax(WL[5], 0.0);
        WR[5] = vac_r ? c.rhoa_floor : fmax(WR[5], 0.0);
    }
    // face velocity (Sec. 4): mean generator velocity plus the correction for
    // the face centroid lying off the generators' midpoint
    const double rix = pos[i], riy = pos[n + i], riz = pos[2 * n + i];
    const double rjx = pos[j] + ox, rjy = pos[n + j] + oy, rjz = pos[2 * n + j] + oz;
    const double drgx = rjx - rix, drgy = rjy - riy, drgz = rjz - riz;
    const double wix = w[i], wiy = w[n + i], wiz = w[2 * n + i];
    const double wjx = w[j], wjy = w[n + j], wjz = w[2 * n + j];
    const double il2 = 1.0 / (drgx * drgx + drgy * drgy + drgz * drgz);
    const double corr = ((wix - wjx) * (fx - 0.5 * (rix + rjx)) + (wiy - wjy) * (fy - 0.5 * (riy + rjy)) +
                         (wiz - wjz) * (fz - 0.5 * (riz + rjz))) * il2;
    const double wfx = corr * drgx + 0.5 * (wix + wjx);
    const double wfy = corr * drgy + 0.5 * (wiy + wjy);
    const double wfz = corr * drgz + 0.5 * (wiz + wjz);
    // primitives, boosted into the face frame (pressure is frame independent)
    const double gm1 = c.gamma - 1.0;
    FaceState L, R;
    {
        const double ir = irl;
        L.rho = WL[0];
        L.irho = ir;
        L.P = gm1 * (WL[4] - kel);
        L.vx = WL[1] * ir - wfx; L.vy = WL[2] * ir - wfy; L.vz = WL[3] * ir - wfz;
    }
    {
        const double ir = irr;
        R.rho = WR[0];
        R.irho = ir;
        R.P = gm1 * (WR[4] - ker);
        R.vx = WR[1] * ir - wfx; R.vy = WR[2] * ir - wfy; R.vz = WR[3] * ir - wfz;
    }
    double F[5];
    WavesT<double> wv;
    riemann_t<double>(c.riemann, L, R, nx, ny, nz, c.gamma, c.igm1, F, NG == 6 ? &wv : nullptr);
    // back to the lab frame: p -> p + m w, E -> E + p.w + |w|^2/2 m
    const double A = m.area[f];
    const double fm = F[0];
    const double fe = F[4] + F[1] * wfx + F[2] * wfy + F[3] * wfz + 0.5 * (wfx * wfx + wfy * wfy + wfz * wfz) * fm;
    flux[f] = A * fm;
    flux[fs + f] = A * (F[1] + fm * wfx);
    flux[2 * fs + f] = A * (F[2] + fm * wfy);
    flux[3 * fs + f] = A * (F[3] + fm * wfz);
    flux[4 * fs + f] = A * fe;
    if constexpr (NG == 6) {
        double mach;
        const double f5 = passive_flux_t<double>(c.riemann, L, R, wv, c.kmach, WL[5], WR[5], fm, mach);
        flux[5 * fs + f] = A * f5;
        flux[6 * fs + f] = mach;
        flux[7 * fs + f] = A * (wfx * nx + wfy * ny + wfz * nz);
    }
}

void launch_face_flux(const MeshDev &m, const HydroCfg &c, const double *pos, const double *w, const double *Wh,
                      const double *grad, double *flux, cudaStream_t s)
{
    const int64_t nfl = face_launch_count(m);
    if (nfl == 0) return;
    int nb = (int)((nfl + 127) / 128);
    if (c.entropy) k_face_flux<6><<<nb, 128, 0, s>>>(m, c, pos, w, Wh, grad, flux);
    else k_face_flux<5><<<nb, 128, 0, s>>>(m, c, pos, w, Wh, grad, flux);
}

// ---------------------------------------------------------------------------
// Conservative update: U_i -= dt sum_{f in i} (+/-) Phi_f, then floors
// ---------------------------------------------------------------------------
// With NG = 6 (Sec. 4.3): a cell whose largest face shock Mach number is
// below mach_th takes E from its entropy, E = |p|^2/(2m) + A rho^gamma V' /
// (gamma - 1); elsewhere (and wherever the floors act) the entropy is reset
// from E.  V' = V + dt sum (+/-) A (w_f . n) is the volume the moving faces
// sweep the cell to in the step.
template <int NG>
__global__ void __launch_bounds__(256) k_update(MeshDev m, HydroCfg c, const double *__restrict__ flux,
                                                const double *__restrict__ dtp, double *__restrict__ U)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n, nf = m.fs;  // flux rows are face-capacity apart
    if (t >= n) return;
    const int64_t i = cell_of(m, t);
    double acc[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) acc[k] = 0.0;
    double mc = 0.0, dv = 0.0;
    for (int e = m.inc_off[i]; e < m.inc_off[i + 1]; ++e) {
        int f = m.inc_face[e];
        double sg = 1.0;
        if (f < 0) { f = ~f; sg = -1.0; }
#pragma unroll
        for (int k = 0; k < NG; ++k) acc[k] += sg * flux[k * nf + f];
        if constexpr (NG == 6) {
            mc = fmax(mc, flux[6 * nf + f]);
            dv += sg * flux[7 * nf + f];
        }
    }
    const double dt = dtp[m.cbox[i]];
    double Un[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) Un[k] = U[k * n + i] - dt * acc[k];
    const double V = m.vol[i], iv = 1.0 / V;
    const double g = c.gamma;
    bool energy = true;
    double Vn = V;
    if constexpr (NG == 6) {
        Vn = V + dt * dv;
        energy = mc >= c.mach_th;
        if (!energy) {
            if (Un[0] > 0.0 && Un[5] > 0.0 && Vn > 0.0) {
                const double rho = Un[0] / Vn;
                const double P = (Un[5] / Un[0]) * pow(rho, g);
                Un[4] = 0.5 * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]) / Un[0] + P * Vn / (g - 1.0);
            } else {
                energy = true;
            }
        }
    }
    double W[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) W[k] = Un[k] * iv;
    const bool ch = apply_floor(W, c.rho_floor, c.eps_floor);
    if (ch) {
#pragma unroll
        for (int k = 0; k < 5; ++k) Un[k] = W[k] * V;
    }
    if constexpr (NG == 6) {
        if (energy || ch) {
            const double Vr = Vn > 0.0 ? Vn : V;
            const double rho = Un[0] / Vr;
            const double P = (g - 1.0) * (Un[4] - 0.5 * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]) / Un[0]) / Vr;
            Un[5] = Un[0] * P / pow(rho, g);
        }
    }
#pragma unroll
    for (int k = 0; k < NG; ++k) U[k * n + i] = Un[k];
}

void launch_update(const MeshDev &m, const HydroCfg &c, const double *flux, const double *dt, double *U,
                   cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    if (c.entropy) k_update<6><<<nb, 256, 0, s>>>(m, c, flux, dt, U);
    else k_update<5><<<nb, 256, 0, s>>>(m, c, flux, dt, U);
}

// ---------------------------------------------------------------------------
// Heun's method (second-order time integration, Sec. 6): per-volume states of
// a stage, and the final average U = (U^n + U**) / 2 with the cell floors on
// the end-of-step mesh.
// ---------------------------------------------------------------------------
template <int NG>
__global__ void __launch_bounds__(256) k_states(MeshDev m, const double *__restrict__ U, double *__restrict__ W)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (i >= n) return;
    const double iv = 1.0 / m.vol[i];
#pragma unroll
    for (int k = 0; k < NG; ++k) W[k * n + i] = U[k * n + i] * iv;
}

void launch_states(const MeshDev &m, const HydroCfg &c, const double *U, double *W, cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    if (c.entropy) k_states<6><<<nb, 256, 0, s>>>(m, U, W);
    else k_states<5><<<nb, 256, 0, s>>>(m, U, W);
}

__global__ void __launch_bounds__(256) k_heun_average(MeshDev m, HydroCfg c, const double *__restrict__ U0,
                                                      double *__restrict__ U)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (i >= n) return;
    const double V = m.vol[i], iv = 1.0 / V;
    double Un[5], W[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        Un[k] = 0.5 * (U0[k * n + i] + U[k * n + i]);
        W[k] = Un[k] * iv;
    }
    if (apply_floor(W, c.rho_floor, c.eps_floor)) {
#pragma unroll
        for (int k = 0; k < 5; ++k) Un[k] = W[k] * V;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k * n + i] = Un[k];
}

void launch_heun_average(const MeshDev &m, const HydroCfg &c, const double *U0, double *U, cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    k_heun_average<<<nb, 256, 0, s>>>(m, c, U0, U);
}

// ---------------------------------------------------------------------------
// Mesh velocity (Sec. 4.2) fused with the per-cell CFL timestep and its
// minimum over each box.  Positive doubles order like their bit patterns, so
// the minimum is an unsigned 64-bit atomicMin: exact and order independent.
// ---------------------------------------------------------------------------
// Minimum of v over the lanes of each box: one atomic per warp when the warp
// lies in one box (cells of a box are contiguous), one per lane otherwise.
__device__ __forceinline__ void box_min(unsigned long long *bits, int box, double v)
{
    const int b0 = __shfl_sync(FULL_MASK_HYDRO, box, 0);
    if (__all_sync(FULL_MASK_HYDRO, box == b0 || box < 0)) {
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL_MASK_HYDRO, v, o));
        if ((threadIdx.x & 31) == 0 && b0 >= 0 && v > 0.0)
            atomicMin(bits + b0, (unsigned long long)__double_as_longlong(v));
    } else if (box >= 0 && v > 0.0) {
        atomicMin(bits + box, (unsigned long long)__double_as_longlong(v));
    }
}
__device__ __forceinline__ double sound_speed(const double W[5], double gamma)
{
    const double ke = 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0];
    double P = (gamma - 1.0) * (W[4] - ke);
    if (P < 0.0) P = 0.0;
    return sqrt(gamma * P / W[0]);
}

__global__ void __launch_bounds__(256) k_mesh_velocity(MeshDev m, HydroCfg c, const double *__restrict__ pos,
                                                       const double *__restrict__ U, double *__restrict__ w,
                                                       unsigned long long *__restrict__ dt_bits)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    double dti = __longlong_as_double(0x7ff0000000000000LL);
    if (i < n) {
        const double V = m.vol[i];
        double W[5];
        load5(U, n, i, 1.0 / V, W);
        const double irm = 1.0 / U[i];  // one division for the three velocity components
        const double vx = U[n + i] * irm, vy = U[2 * n + i] * irm, vz = U[3 * n + i] * irm;
        double wx = c.eta * vx, wy = c.eta * vy, wz = c.eta * vz;
        const double cs = sound_speed(W, c.gamma);
        const double R = cbrt(3.0 * V / (4.0 * 3.14159265358979323846));
        if (c.regularize) {
            const double dx = m.cen[i] - pos[i], dy = m.cen[n + i] - pos[n + i], dz = m.cen[2 * n + i] - pos[2 * n + i];
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double zr = c.zeta * R;
            double ramp = 0.0;
            if (d > 1.1 * zr) ramp = 1.0;
            else if (d >= 0.9 * zr) ramp = (d - 0.9 * zr) / (0.2 * zr);
            if (ramp > 0.0 && d > 0.0) {
                const double s = c.chi * cs * ramp / d;
                wx += s * dx; wy += s * dy; wz += s * dz;
            }
        }
        if (w) { w[i] = wx; w[n + i] = wy; w[2 * n + i] = wz; }
        const double rx = vx - wx, ry = vy - wy, rz = vz - wz;
        dti = c.cfl * R / (cs + sqrt(rx * rx + ry * ry + rz * rz));
    }
    if (dt_bits) box_min(dt_bits, i < n ? m.cbox[i] : -1, dti);
}

// CFL timestep for a given generator velocity w (Sec. 4.2).
__global__ void __launch_bounds__(256) k_timestep(MeshDev m, HydroCfg c, const double *__restrict__ U,
                                                  const double *__restrict__ w, unsigned long long *__restrict__ dt_bits)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    double dti = __longlong_as_double(0x7ff0000000000000LL);
    if (i < n) {
        const double V = m.vol[i];
        double W[5];
        load5(U, n, i, 1.0 / V, W);
        const double rx = U[n + i] / U[i] - w[i], ry = U[2 * n + i] / U[i] - w[n + i], rz = U[3 * n + i] / U[i] - w[2 * n + i];
        const double R = cbrt(3.0 * V / (4.0 * 3.14159265358979323846));
        dti = c.cfl * R / (sound_speed(W, c.gamma) + sqrt(rx * rx + ry * ry + rz * rz));
    }
    box_min(dt_bits, i < n ? m.cbox[i] : -1, dti);
}

void launch_timestep(const MeshDev &m, const HydroCfg &c, const double *U, const double *w, double *dt_min,
                     cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    k_timestep<<<nb, 256, 0, s>>>(m, c, U, w, reinterpret_cast<unsigned long long *>(dt_min));
}

__global__ void k_dt_init(double *dt, int nbox)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) dt[b] = __longlong_as_double(0x7ff0000000000000LL);
}

void launch_dt_init(double *dt, int nbox, cudaStream_t s) { k_dt_init<<<(nbox + 255) / 256, 256, 0, s>>>(dt, nbox); }

void launch_mesh_velocity(const MeshDev &m, const HydroCfg &c, const double *pos, const double *U, double *w,
                          double *dt_min, cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    k_mesh_velocity<<<nb, 256, 0, s>>>(m, c, pos, U, w, reinterpret_cast<unsigned long long *>(dt_min));
}

// ---------------------------------------------------------------------------
// Drift: r += w dt wrapped into [0, L)
// ---------------------------------------------------------------------------
__global__ void k_drift(double *__restrict__ pos, int64_t n, const double *__restrict__ w,
                        const double *__restrict__ dtp, const int *__restrict__ cbox, const double *__restrict__ boxL)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = cbox[i];
    const double dt = dtp[b];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double L = boxL[3 * b + d];
        double x = fmod(pos[d * n + i] + w[d * n + i] * dt, L);
        if (x < 0.0) x += L;
        if (x >= L) x -= L;
        pos[d * n + i] = x;
    }
}

void launch_drift(double *pos, int64_t n, const double *w, const double *dt, const int *cbox, const double *boxL,
                  cudaStream_t s)
{
    int nb = (int)((n + 255) / 256);
    k_drift<<<nb, 256, 0, s>>>(pos, n, w, dt, cbox, boxL);
}

// ---------------------------------------------------------------------------
// Charges from primitives, and compensated totals
// ---------------------------------------------------------------------------
__global__ void k_prims_to_charges(MeshDev m, HydroCfg c, const double *__restrict__ rho, const double *__restrict__ vel,
                                   const double *__restrict__ P, double *__restrict__ U)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (i >= n) return;
    const double V = m.vol[i], r = rho[i];
    const double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
    U[i] = r * V;
    U[n + i] = r * vx * V;
    U[2 * n + i] = r * vy * V;
    U[3 * n + i] = r * vz * V;
    U[4 * n + i] = (P[i] / (c.gamma - 1.0) + 0.5 * r * (vx * vx + vy * vy + vz * vz)) * V;
    if (c.entropy) U[5 * n + i] = (r * V) * P[i] / pow(r, c.gamma);  // m A, A = P / rho^gamma (Sec. 4.3)
}

void launch_prims_to_charges(const MeshDev &m, const HydroCfg &c, const double *rho, const double *vel,
                             const double *P, double *U, cudaStream_t s)
{
    int nb = (int)((m.n + 255) / 256);
    k_prims_to_charges<<<nb, 256, 0, s>>>(m, c, rho, vel, P, U);
}

// Neumaier sum pair (s, comp): value = s + comp.
__device__ __forceinline__ void neumaier_add(double &s, double &comp, double x)
{
    const double t = s + x;
    if (fabs(s) >= fabs(x)) comp += (s - t) + x;
    else comp += (x - t) + s;
    s = t;
}

// Each block reduces a contiguous range per component with a Neumaier sum
// per thread and a fixed-order tree over threads; a second pass sums the
// block partials in order.  Deterministic for a given launch shape.
__global__ void k_totals_partial(const double *__restrict__ U, int64_t n, double *__restrict__ partial)
{
    __shared__ double ss[256], sc[256];
    const int nblk = gridDim.x;
    const int64_t per = (n + nblk - 1) / nblk;
    const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
    for (int k = 0; k < 5; ++k) {
        double s = 0.0, cmp = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) neumaier_add(s, cmp, U[k * n + i]);
        ss[threadIdx.x] = s;
        sc[threadIdx.x] = cmp;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                double a = ss[threadIdx.x], ca = sc[threadIdx.x];
                neumaier_add(a, ca, ss[threadIdx.x + o]);
                ca += sc[threadIdx.x + o];
                ss[threadIdx.x] = a;
                sc[threadIdx.x] = ca;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            partial[2 * (k * nblk + blockIdx.x)] = ss[0];
            partial[2 * (k * nblk + blockIdx.x) + 1] = sc[0];
        }
        __syncthreads();
    }
}

__global__ void k_totals_final(const double *__restrict__ partial, int nblk, double *__restrict__ totals)
{
    const int k = threadIdx.x;
    if (k >= 5) return;
    double s = 0.0, cmp = 0.0;
    for (int b = 0; b < nblk; ++b) {
        neumaier_add(s, cmp, partial[2 * (k * nblk + b)]);
        cmp += partial[2 * (k * nblk + b) + 1];
    }
    totals[k] = s + cmp;
}

void launch_totals(const double *U, int64_t n, double *partial, int nblocks, double *totals, cudaStream_t s)
{
    k_totals_partial<<<nblocks, 256, 0, s>>>(U, n, partial);
    k_totals_final<<<1, 32, 0, s>>>(partial, nblocks, totals);
}

// The cell order of MeshDev::order: each block sorts its CELL_ORDER_BLOCK
// cells by incident-face count (ties by index: a stable, deterministic order)
// by counting, for each cell, the block's cells that come before it.
__global__ void __launch_bounds__(CELL_ORDER_BLOCK) k_cell_order(int64_t n, const int *__restrict__ inc_off,
                                                                 int *__restrict__ order)
{
    __shared__ int cnt[CELL_ORDER_BLOCK];
    const int64_t base = (int64_t)blockIdx.x * CELL_ORDER_BLOCK;
    const int t = threadIdx.x;
    const int64_t i = base + t;
    const int c = i < n ? inc_off[i + 1] - inc_off[i] : 0x7fffffff;  // beyond n: last
    cnt[t] = c;
    __syncthreads();
    int rank = 0;
    for (int u = 0; u < CELL_ORDER_BLOCK; ++u) {
        const int cu = cnt[u];
        rank += (cu < c) || (cu == c && u < t);
    }
    if (i < n) order[base + rank] = (int)i;
}

void launch_cell_order(int64_t n, const int *inc_off, int *order, cudaStream_t s)
{
    const int64_t nb = (n + CELL_ORDER_BLOCK - 1) / CELL_ORDER_BLOCK;
    k_cell_order<<<(unsigned)nb, CELL_ORDER_BLOCK, 0, s>>>(n, inc_off, order);
}

}  // namespace mm
