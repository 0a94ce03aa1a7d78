// mm_hydro32.cu -- the mixed-precision finite-volume stages (precision = 1).
//
// Gradients, limiters, the half step, the reconstruction and the face-frame
// HLLC run in FP32 with FP32 accumulation; the charge update accumulates the
// FP32 face fluxes in FP64 and updates the FP64 charges (Sec. 4, 4.1).  Every
// position-like quantity enters FP32 as a short difference formed in FP64:
// the neighbour offset q = r_j + s L - r_i, the face centroid relative to r_i
// and the cell centroid relative to its generator, so FP32 keeps ~1e-7 of
// their own size rather than of the box size.
//
// Records (16-byte vectors, one or two sectors per gather):
//   face  f: ij = (i, j); fa = (A, n); fq = (q, x_f - r_i .x); ff = (x_f - r_i .y, .z)
//   cell  i: rec[2i] = (W0..W3), rec[2i+1] = (W4, c_i - r_i)      (W^n and W^(n+1/2))
//            grad[4i..4i+3] = 15 slopes (row 3k+d = dW_k/dx_d) + pad
//            wv[i] = (w, 0)
//   flux  f: flux[2f] = (F0..F3), flux[2f+1] = (F4, 0, 0, 0)     (A F, lab frame)
#include "mm_internal.cuh"
#include "mm_riemann.cuh"

namespace mm {

__device__ __forceinline__ void decode_shift32(int code, double &sx, double &sy, double &sz)
{
    sx = (double)(code % 3 - 1);
    sy = (double)((code / 3) % 3 - 1);
    sz = (double)(code / 9 - 1);
}

__global__ void __launch_bounds__(256) k_faces32(MeshDev m, const double *__restrict__ pos, Mixed x)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= face_count(m)) return;
    const int64_t n = m.n, fs = m.fs;
    const int i = m.face_i[f], j = m.face_j[f];
    double sx, sy, sz;
    decode_shift32(m.face_shift[f], sx, sy, sz);
    const double *L = m.boxL + 3 * m.cbox[i];
    const double qx = pos[j] + sx * L[0] - pos[i];
    const double qy = pos[n + j] + sy * L[1] - pos[n + i];
    const double qz = pos[2 * n + j] + sz * L[2] - pos[2 * n + i];
    const double fx = m.fcen[f] - pos[i], fy = m.fcen[fs + f] - pos[n + i], fz = m.fcen[2 * fs + f] - pos[2 * n + i];
    x.fij[f] = make_int2(i, j);
    x.fa[f] = make_float4((float)m.area[f], (float)m.normal[f], (float)m.normal[fs + f], (float)m.normal[2 * fs + f]);
    x.fq[f] = make_float4((float)qx, (float)qy, (float)qz, (float)fx);
    x.ff[f] = make_float2((float)fy, (float)fz);
}

__global__ void __launch_bounds__(256) k_pack32(MeshDev m, const double *__restrict__ U, const double *__restrict__ pos,
                                                const double *__restrict__ w, Mixed x)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (i >= n) return;
    const double iv = 1.0 / m.vol[i];
    x.cw[2 * i] = make_float4((float)(U[i] * iv), (float)(U[n + i] * iv), (float)(U[2 * n + i] * iv),
                              (float)(U[3 * n + i] * iv));
    x.cw[2 * i + 1] = make_float4((float)(U[4 * n + i] * iv), (float)(m.cen[i] - pos[i]),
                                  (float)(m.cen[n + i] - pos[n + i]), (float)(m.cen[2 * n + i] - pos[2 * n + i]));
    x.wv[i] = make_float4((float)w[i], (float)w[n + i], (float)w[2 * n + i], 0.0f);
}

struct Nbr32 {
    int f, o;
    float sg;
};

__device__ __forceinline__ Nbr32 nbr32(const MeshDev &m, const Mixed &x, int e)
{
    Nbr32 r;
    int f = m.inc_face[e];
    const bool fwd = f >= 0;
    if (!fwd) f = ~f;
    const int2 ij = x.fij[f];
    r.f = f;
    r.o = fwd ? ij.y : ij.x;
    r.sg = fwd ? 1.0f : -1.0f;
    return r;
}

// Limited gradient in FP32 (same estimator and limiters as the FP64 path);
// with PREDICT the half step is taken and W^(n+1/2) written instead.
template <bool PREDICT>
// six resident blocks (80 registers): left free, ptxas trades a spill for a seventh
__global__ void __launch_bounds__(128, 6) k_gradient32(MeshDev m, HydroCfg c, Mixed x, const float4 *__restrict__ rin,
                                                    float4 *__restrict__ rout, const double *__restrict__ dtp)
{
    // index order: this kernel is bound by its gathers, and the FP32 loop's
    // uneven lengths cost less than scattering the cells of a warp
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (i >= n) return;
    const float4 a0 = rin[2 * i], a1 = rin[2 * i + 1];
    const float Wi[5] = {a0.x, a0.y, a0.z, a0.w, a1.x};
    const float dix = a1.y, diy = a1.z, diz = a1.w;
    const int e0 = m.inc_off[i], e1 = m.inc_off[i + 1];
    float M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    float b[15];
    float wmax[5], wmin[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) { wmax[k] = Wi[k]; wmin[k] = Wi[k]; }
#pragma unroll
    for (int k = 0; k < 15; ++k) b[k] = 0.0f;
    for (int e = e0; e < e1; ++e) {
        const Nbr32 q = nbr32(m, x, e);
        const float4 fa = x.fa[q.f], fq = x.fq[q.f];
        const float4 o0 = rin[2 * q.o], o1 = rin[2 * q.o + 1];
        const float ha = 0.5f * fa.x;
        const float ax = ha * q.sg * fa.y, ay = ha * q.sg * fa.z, az = ha * q.sg * fa.w;
        const float dx = q.sg * fq.x + o1.y - dix, dy = q.sg * fq.y + o1.z - diy, dz = q.sg * fq.z + o1.w - diz;
        M[0] += ax * dx; M[1] += ax * dy; M[2] += ax * dz;
        M[3] += ay * dx; M[4] += ay * dy; M[5] += ay * dz;
        M[6] += az * dx; M[7] += az * dy; M[8] += az * dz;
        const float Wo[5] = {o0.x, o0.y, o0.z, o0.w, o1.x};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float dw = Wo[k] - Wi[k];
            b[3 * k + 0] += ax * dw;
            b[3 * k + 1] += ay * dw;
            b[3 * k + 2] += az * dw;
            wmax[k] = fmaxf(wmax[k], Wo[k]);
            wmin[k] = fminf(wmin[k], Wo[k]);
        }
    }
    const float c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const float c10 = M[2] * M[7] - M[1] * M[8], c11 = M[0] * M[8] - M[2] * M[6], c12 = M[1] * M[6] - M[0] * M[7];
    const float c20 = M[1] * M[5] - M[2] * M[4], c21 = M[2] * M[3] - M[0] * M[5], c22 = M[0] * M[4] - M[1] * M[3];
    const float idet = 1.0f / (M[0] * c00 + M[1] * c01 + M[2] * c02);
    float g[15];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float b0 = b[3 * k], b1 = b[3 * k + 1], b2 = b[3 * k + 2];
        g[3 * k + 0] = (c00 * b0 + c10 * b1 + c20 * b2) * idet;
        g[3 * k + 1] = (c01 * b0 + c11 * b1 + c21 * b2) * idet;
        g[3 * k + 2] = (c02 * b0 + c12 * b1 + c22 * b2) * idet;
    }
    if (c.limiter >= 1) {
        float dmax[5], dmin[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) { dmax[k] = 0.0f; dmin[k] = 0.0f; }
        for (int e = e0; e < e1; ++e) {
            const Nbr32 q = nbr32(m, x, e);
            const float4 fq = x.fq[q.f];
            const float4 o1 = rin[2 * q.o + 1];
            float dx, dy, dz;
            if (c.limiter == 3) {
                // face centroid relative to this cell's centroid: x_f - r_i - d_i, or x_f - q - r_i - d_j
                const float2 ff = x.ff[q.f];
                const float hx = q.sg > 0.0f ? 0.0f : fq.x, hy = q.sg > 0.0f ? 0.0f : fq.y, hz = q.sg > 0.0f ? 0.0f : fq.z;
                dx = fq.w - hx - dix;
                dy = ff.x - hy - diy;
                dz = ff.y - hz - diz;
            } else {
                dx = q.sg * fq.x + o1.y - dix;
                dy = q.sg * fq.y + o1.z - diy;
                dz = q.sg * fq.z + o1.w - diz;
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float del = g[3 * k] * dx + g[3 * k + 1] * dy + g[3 * k + 2] * dz;
                dmax[k] = fmaxf(dmax[k], del);
                dmin[k] = fminf(dmin[k], del);
            }
        }
        float al[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            al[k] = 1.0f;
            if (dmax[k] > 0.0f) al[k] = fminf(al[k], (wmax[k] - Wi[k]) / dmax[k]);
            if (dmin[k] < 0.0f) al[k] = fminf(al[k], (wmin[k] - Wi[k]) / dmin[k]);
        }
        if (c.limiter == 2) {
            // DM with the unlimited gradient, over the neighbours whose Delta
            // is nonzero beyond the rounding of g and d (2^-40 |g|_1 |d|_1;
            // toward the equal-valued transverse neighbours of a lattice Delta
            // is zero in exact arithmetic), as a fraction (num, den > 0)
            const float theta = (float)c.theta;
            float rn[5], rd[5], gl[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                rn[k] = 1.0f; rd[k] = 1.0f;
                gl[k] = 0x1p-40f * (fabsf(g[3 * k]) + fabsf(g[3 * k + 1]) + fabsf(g[3 * k + 2]));
            }
            for (int e = e0; e < e1; ++e) {
                const Nbr32 q = nbr32(m, x, e);
                const float4 fq = x.fq[q.f];
                const float4 o0 = rin[2 * q.o], o1 = rin[2 * q.o + 1];
                const float dx = q.sg * fq.x + o1.y - dix, dy = q.sg * fq.y + o1.z - diy, dz = q.sg * fq.z + o1.w - diz;
                const float dl = fabsf(dx) + fabsf(dy) + fabsf(dz);
                const float Wo[5] = {o0.x, o0.y, o0.z, o0.w, o1.x};
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float del = g[3 * k] * dx + g[3 * k + 1] * dy + g[3 * k + 2] * dz;
                    if (!(fabsf(del) > gl[k] * dl)) continue;
                    float num = theta * (Wo[k] - Wi[k]);
                    float den = del;
                    if (den < 0.0f) { num = -num; den = -den; }
                    if (num < 0.0f) num = 0.0f;
                    if (num * rd[k] < rn[k] * den) { rn[k] = num; rd[k] = den; }
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) al[k] *= fminf(1.0f, rn[k] / rd[k]);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            g[3 * k] *= al[k];
            g[3 * k + 1] *= al[k];
            g[3 * k + 2] *= al[k];
        }
    }
    if (!PREDICT) {
        x.grad[4 * i] = make_float4(g[0], g[1], g[2], g[3]);
        x.grad[4 * i + 1] = make_float4(g[4], g[5], g[6], g[7]);
        x.grad[4 * i + 2] = make_float4(g[8], g[9], g[10], g[11]);
        x.grad[4 * i + 3] = make_float4(g[12], g[13], g[14], 0.0f);
        return;
    }
    // half step through the chain rule of the Euler flux on (rho, m, E)
    const float gm1 = (float)c.gamma - 1.0f;
    const float ir = 1.0f / Wi[0];
    const float u[3] = {Wi[1] * ir, Wi[2] * ir, Wi[3] * ir};
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float P = gm1 * (Wi[4] - 0.5f * Wi[0] * u2);
    float dP[3], divu = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float drho = g[d];
        divu += (g[3 * (1 + d) + d] - u[d] * drho) * ir;
        dP[d] = gm1 * (g[12 + d] - (u[0] * g[3 + d] + u[1] * g[6 + d] + u[2] * g[9 + d]) + 0.5f * u2 * drho);
    }
    float rate[5];
    rate[0] = -(g[3] + g[7] + g[11]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) s += u[d] * g[3 * (1 + k) + d];
        rate[1 + k] = -(s + Wi[1 + k] * divu) - dP[k];
    }
    {
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) s += u[d] * (g[12 + d] + dP[d]);
        rate[4] = -(s + (Wi[4] + P) * divu);
    }
    const float hdt = 0.5f * (float)dtp[m.cbox[i]];
    rout[2 * i] = make_float4(Wi[0] + hdt * rate[0], Wi[1] + hdt * rate[1], Wi[2] + hdt * rate[2], Wi[3] + hdt * rate[3]);
    rout[2 * i + 1] = make_float4(Wi[4] + hdt * rate[4], dix, diy, diz);
}

__global__ void __launch_bounds__(128) k_face_flux32(MeshDev m, HydroCfg c, Mixed x)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= face_count(m)) return;
    const int2 ij = x.fij[f];
    const int i = ij.x, j = ij.y;
    const float4 fa = x.fa[f], fq = x.fq[f];
    const float2 ff = x.ff[f];
    const float qx = fq.x, qy = fq.y, qz = fq.z;           // r_j' - r_i
    const float fx = fq.w, fy = ff.x, fz = ff.y;           // x_f - r_i
    const float4 hi0 = x.ch[2 * i], hi1 = x.ch[2 * i + 1];
    const float4 hj0 = x.ch[2 * j], hj1 = x.ch[2 * j + 1];
    const float dlx = fx - hi1.y, dly = fy - hi1.z, dlz = fz - hi1.w;                // x_f - c_i
    const float drx = fx - qx - hj1.y, dry = fy - qy - hj1.z, drz = fz - qz - hj1.w; // x_f - c_j'
    float WL[5] = {hi0.x, hi0.y, hi0.z, hi0.w, hi1.x};
    float WR[5] = {hj0.x, hj0.y, hj0.z, hj0.w, hj1.x};
    {
        float gi[16], gj[16];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 a = x.grad[4 * i + r], bq = x.grad[4 * j + r];
            gi[4 * r] = a.x; gi[4 * r + 1] = a.y; gi[4 * r + 2] = a.z; gi[4 * r + 3] = a.w;
            gj[4 * r] = bq.x; gj[4 * r + 1] = bq.y; gj[4 * r + 2] = bq.z; gj[4 * r + 3] = bq.w;
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            WL[k] += dlx * gi[3 * k] + dly * gi[3 * k + 1] + dlz * gi[3 * k + 2];
            WR[k] += drx * gj[3 * k] + dry * gj[3 * k + 1] + drz * gj[3 * k + 2];
        }
    }
    const float rf = (float)c.rho_floor, ef = (float)c.eps_floor;
    float irl, irr, kel, ker;
    apply_floor_ir_t<float>(WL, rf, ef, irl, kel);
    apply_floor_ir_t<float>(WR, rf, ef, irr, ker);
    // face velocity (Sec. 4)
    const float4 wi = x.wv[i], wj = x.wv[j];
    const float mx = fx - 0.5f * qx, my = fy - 0.5f * qy, mz = fz - 0.5f * qz;
    const float corr = ((wi.x - wj.x) * mx + (wi.y - wj.y) * my + (wi.z - wj.z) * mz) / (qx * qx + qy * qy + qz * qz);
    const float wfx = corr * qx + 0.5f * (wi.x + wj.x);
    const float wfy = corr * qy + 0.5f * (wi.y + wj.y);
    const float wfz = corr * qz + 0.5f * (wi.z + wj.z);
    const float gam = (float)c.gamma, gm1 = gam - 1.0f;
    FaceStateT<float> L, R;
    {
        const float ir = irl;
        L.rho = WL[0];
        L.irho = ir;
        L.P = gm1 * (WL[4] - kel);
        L.vx = WL[1] * ir - wfx; L.vy = WL[2] * ir - wfy; L.vz = WL[3] * ir - wfz;
    }
    {
        const float ir = irr;
        R.rho = WR[0];
        R.irho = ir;
        R.P = gm1 * (WR[4] - ker);
        R.vx = WR[1] * ir - wfx; R.vy = WR[2] * ir - wfy; R.vz = WR[3] * ir - wfz;
    }
    float F[5];
    riemann_t<float>(c.riemann, L, R, fa.y, fa.z, fa.w, gam, 1.0f / gm1, F);
    const float A = fa.x, fm = F[0];
    const float fe = F[4] + F[1] * wfx + F[2] * wfy + F[3] * wfz + 0.5f * (wfx * wfx + wfy * wfy + wfz * wfz) * fm;
    x.flux[2 * f] = make_float4(A * fm, A * (F[1] + fm * wfx), A * (F[2] + fm * wfy), A * (F[3] + fm * wfz));
    x.flux[2 * f + 1] = make_float4(A * fe, 0.0f, 0.0f, 0.0f);
}

// FP64 charge update from the FP32 face fluxes: each flux enters both cells
// as the same value with opposite signs, so the totals are conserved to the
// rounding of the FP64 sums.
__global__ void __launch_bounds__(256) k_update32(MeshDev m, HydroCfg c, Mixed x, const double *__restrict__ dtp,
                                                  double *__restrict__ U)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = m.n;
    if (t >= n) return;
    const int64_t i = cell_of(m, t);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int e = m.inc_off[i]; e < m.inc_off[i + 1]; ++e) {
        int f = m.inc_face[e];
        const double sg = f >= 0 ? 1.0 : -1.0;
        if (f < 0) f = ~f;
        const float4 a = x.flux[2 * f], bq = x.flux[2 * f + 1];
        acc[0] += sg * (double)a.x;
        acc[1] += sg * (double)a.y;
        acc[2] += sg * (double)a.z;
        acc[3] += sg * (double)a.w;
        acc[4] += sg * (double)bq.x;
    }
    const double dt = dtp[m.cbox[i]];
    double Un[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Un[k] = U[k * n + i] - dt * acc[k];
    const double V = m.vol[i], iv = 1.0 / V;
    double W[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) W[k] = Un[k] * iv;
    if (apply_floor_t<double>(W, c.rho_floor, c.eps_floor)) {
#pragma unroll
        for (int k = 0; k < 5; ++k) Un[k] = W[k] * V;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k * n + i] = Un[k];
}

void launch_mixed_step(const MeshDev &m, const HydroCfg &c, const double *pos, const double *w, const double *dt,
                       Mixed x, double *U, cudaStream_t s, void (*mark)(void *, int, bool), void *mark_arg)
{
    const int nbc = (int)((m.n + 127) / 128), nbc2 = (int)((m.n + 255) / 256);
    const int64_t nfl = face_launch_count(m);
    const int nbf = (int)((nfl + 255) / 256), nbf2 = (int)((nfl + 127) / 128);
    mark(mark_arg, MM_STAGE_GRADIENT_HALF, true);
    if (nfl > 0) k_faces32<<<nbf, 256, 0, s>>>(m, pos, x);
    k_pack32<<<nbc2, 256, 0, s>>>(m, U, pos, w, x);
    k_gradient32<true><<<nbc, 128, 0, s>>>(m, c, x, x.cw, x.ch, dt);
    mark(mark_arg, MM_STAGE_GRADIENT_HALF, false);
    mark(mark_arg, MM_STAGE_GRADIENT, true);
    k_gradient32<false><<<nbc, 128, 0, s>>>(m, c, x, x.ch, nullptr, dt);
    mark(mark_arg, MM_STAGE_GRADIENT, false);
    mark(mark_arg, MM_STAGE_FACE_FLUX, true);
    if (nfl > 0) k_face_flux32<<<nbf2, 128, 0, s>>>(m, c, x);
    mark(mark_arg, MM_STAGE_FACE_FLUX, false);
    mark(mark_arg, MM_STAGE_UPDATE, true);
    k_update32<<<nbc2, 256, 0, s>>>(m, c, x, dt, U);
    mark(mark_arg, MM_STAGE_UPDATE, false);
}

}  // namespace mm
