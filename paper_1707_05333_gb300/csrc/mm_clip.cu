// mm_clip.cu -- Voronoi cells by half-space clipping, one warp per cell (Sec. 3).
//
// The paper builds each cell by starting from a large box around the
// generator p and cutting it with the bisector plane of every neighbour n,
// nearest first, until |n - p| exceeds twice the distance to the farthest
// vertex.  Here:
//  * The starting box is [-L/2, L/2]^3 about p: its six faces are the
//    bisectors with p's own periodic images, so the true cell lies inside.
//  * The cell is kept as its dual: every vertex is a triangle (a,b,c) of
//    plane indices, oriented so det(q_a, q_b, q_c) > 0; its position is the
//    intersection of those three planes, solved in FP64.  A cut removes the
//    triangles beyond the plane; the directed edges of removed triangles
//    whose reverse edge is not also removed form the rim of the hole, and
//    each rim edge x->y becomes a new triangle (x, y, k).  A 64x64 bit
//    matrix in shared memory answers "is y->x removed" in O(1).
//  * Candidates come from a uniform grid of bins, ring by ring (Chebyshev
//    distance in bins), filtered by |q| < 2 r_max, sorted by (|q|, id,
//    image) with a warp bitonic sort, and clipped in that order.  The cell
//    is complete once 2 r_max is inside the radius the gathered rings are
//    guaranteed to cover.
//  * Geometry: a face's polygon is walked around its plane in the dual, its
//    area and centroid come from a fan, and the cell volume and centroid
//    from the pyramids (apex p) over the faces: V_f = A h / 3 with h = |q|/2,
//    centroid 3/4 of the way from p to the face centroid.
#include "mm_internal.cuh"

namespace mm {

constexpr unsigned FULL = 0xffffffffu;
constexpr int CBATCH = 64;  // candidate buffer; flushed (sorted + clipped) when full

struct ClipSmem {
    double cx[CBATCH], cy[CBATCH], cz[CBATCH], cd[CBATCH];  // candidates: q and |q|^2
    int cid[CBATCH], csh[CBATCH];
    double px[PMAX], py[PMAX], pz[PMAX], po[PMAX];  // planes x.q <= po
    int pnb[PMAX], psh[PMAX];
    double tx[TMAX], ty[TMAX], tz[TMAX];  // vertices
    unsigned tv[TMAX];                    // a | b << 8 | c << 16
    unsigned long long bm[PMAX];          // removed directed edges x -> y
    unsigned stage[NSTAGE];               // triangles created by the current cut
    // per-plane face results, written during finalisation
    double fa[PMAX], fcx[PMAX], fcy[PMAX], fcz[PMAX];
};

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(FULL, v, o);
    return v;
}

// Intersection of planes a, b, c: x = (o_a (q_b x q_c) + o_b (q_c x q_a) + o_c (q_a x q_b)) / det.
__device__ __forceinline__ void plane_vertex(const ClipSmem &S, int a, int b, int c, double &x, double &y,
                                             double &z)
{
    const double ax = S.px[a], ay = S.py[a], az = S.pz[a], ao = S.po[a];
    const double bx = S.px[b], by = S.py[b], bz = S.pz[b], bo = S.po[b];
    const double cx = S.px[c], cy = S.py[c], cz = S.pz[c], co = S.po[c];
    const double bcx = by * cz - bz * cy, bcy = bz * cx - bx * cz, bcz = bx * cy - by * cx;
    const double cax = cy * az - cz * ay, cay = cz * ax - cx * az, caz = cx * ay - cy * ax;
    const double abx = ay * bz - az * by, aby = az * bx - ax * bz, abz = ax * by - ay * bx;
    const double inv = 1.0 / (ax * bcx + ay * bcy + az * bcz);
    x = (ao * bcx + bo * cax + co * abx) * inv;
    y = (ao * bcy + bo * cay + co * aby) * inv;
    z = (ao * bcz + bo * caz + co * abz) * inv;
}

// Candidate order: (|q|^2, id, image code).
__device__ __forceinline__ bool cand_less(const ClipSmem &S, int a, int b)
{
    if (S.cd[a] != S.cd[b]) return S.cd[a] < S.cd[b];
    if (S.cid[a] != S.cid[b]) return S.cid[a] < S.cid[b];
    return S.csh[a] < S.csh[b];
}

__device__ __forceinline__ void cand_swap(ClipSmem &S, int a, int b)
{
    double t;
    t = S.cx[a]; S.cx[a] = S.cx[b]; S.cx[b] = t;
    t = S.cy[a]; S.cy[a] = S.cy[b]; S.cy[b] = t;
    t = S.cz[a]; S.cz[a] = S.cz[b]; S.cz[b] = t;
    t = S.cd[a]; S.cd[a] = S.cd[b]; S.cd[b] = t;
    int u;
    u = S.cid[a]; S.cid[a] = S.cid[b]; S.cid[b] = u;
    u = S.csh[a]; S.csh[a] = S.csh[b]; S.csh[b] = u;
}

// Warp bitonic sort of the first m candidates (padded to a power of two).
__device__ void sort_candidates(ClipSmem &S, int m, int lane)
{
    int P = 1;
    while (P < m) P <<= 1;
    for (int t = m + lane; t < P; t += 32) {
        S.cd[t] = __longlong_as_double(0x7ff0000000000000LL);  // +inf
        S.cid[t] = 0x7fffffff;
        S.csh[t] = 0x7fffffff;
    }
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < P; t += 32) {
                int u = t ^ j;
                if (u > t) {
                    bool up = (t & k) == 0;
                    if (cand_less(S, u, t) == up) cand_swap(S, t, u);
                }
            }
            __syncwarp();
        }
}

struct CellState {
    int np, nt;
    double rmax2;
    int err;
    int cuts;
};

// Clip the cell by candidate k.  Warp-uniform control flow throughout.
template <int PREC>
__device__ void clip_by(ClipSmem &S, int k, CellState &C, int lane)
{
    const double qx = S.cx[k], qy = S.cy[k], qz = S.cz[k], off = 0.5 * S.cd[k];
    const int nchunk = (C.nt + 31) >> 5;
    unsigned outm[TMAX / 32];
    unsigned anyv = 0;
#pragma unroll
    for (int c = 0; c < TMAX / 32; ++c) {
        bool o = false;
        int t = c * 32 + lane;
        if (c < nchunk && t < C.nt) {
            if (PREC == 0) {
                o = qx * S.tx[t] + qy * S.ty[t] + qz * S.tz[t] > off;
            } else {
                // FP32 filter with a forward error bound; FP64 only near a tie.
                float fx = (float)S.tx[t], fy = (float)S.ty[t], fz = (float)S.tz[t];
                float s = fmaf((float)qx, fx, fmaf((float)qy, fy, fmaf((float)qz, fz, -(float)off)));
                float mag = fabsf((float)qx * fx) + fabsf((float)qy * fy) + fabsf((float)qz * fz) + (float)off;
                if (fabsf(s) > 4.0e-6f * mag) o = s > 0.0f;
                else o = qx * S.tx[t] + qy * S.ty[t] + qz * S.tz[t] > off;
            }
        }
        outm[c] = __ballot_sync(FULL, o);
        anyv |= outm[c];
    }
    if (anyv == 0) return;
    if (C.np >= PMAX) { C.err |= ST_ECAP_PLANE; return; }
    const int kp = C.np;
    if (lane == 0) {
        S.px[kp] = qx; S.py[kp] = qy; S.pz[kp] = qz; S.po[kp] = off;
        S.pnb[kp] = S.cid[k]; S.psh[kp] = S.csh[k];
    }
    // mark the directed edges of the removed triangles
#pragma unroll
    for (int c = 0; c < TMAX / 32; ++c) {
        if ((outm[c] >> lane) & 1u) {
            unsigned v = S.tv[c * 32 + lane];
            unsigned a = v & 255u, b = (v >> 8) & 255u, cc = (v >> 16) & 255u;
            atomicOr(&S.bm[a], 1ull << b);
            atomicOr(&S.bm[b], 1ull << cc);
            atomicOr(&S.bm[cc], 1ull << a);
        }
    }
    __syncwarp();
    // rim edges: removed x->y whose reverse y->x is not removed
    int nnew = 0;
    unsigned long long xs = 0, ys = 0;
#pragma unroll
    for (int c = 0; c < TMAX / 32; ++c) {
        if (outm[c] == 0) continue;  // warp-uniform
        unsigned e[3];
        int cnt = 0;
        if ((outm[c] >> lane) & 1u) {
            unsigned v = S.tv[c * 32 + lane];
            unsigned a = v & 255u, b = (v >> 8) & 255u, cc = (v >> 16) & 255u;
            unsigned ex[3] = {a, b, cc}, ey[3] = {b, cc, a};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (!((S.bm[ey[q]] >> ex[q]) & 1ull)) {
                    e[cnt++] = ex[q] | (ey[q] << 8) | ((unsigned)kp << 16);
                    xs |= 1ull << ex[q];
                    ys |= 1ull << ey[q];
                }
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        int tot = __shfl_sync(FULL, incl, 31);
        int base = nnew + incl - cnt;
        for (int q = 0; q < cnt; ++q)
            if (base + q < NSTAGE) S.stage[base + q] = e[q];
        nnew += tot;
    }
    __syncwarp();
    for (int r = lane; r < C.np; r += 32) S.bm[r] = 0ull;
    xs = warp_or64(xs);
    ys = warp_or64(ys);
    if (nnew > NSTAGE) { C.err |= ST_ECAP_STAGE; return; }
    if (nnew < 3 || xs != ys || __popcll(xs) != nnew) { C.err |= ST_EDEGEN; return; }
    int nrem = 0;
#pragma unroll
    for (int c = 0; c < TMAX / 32; ++c) nrem += __popc(outm[c]);
    const int nkept = C.nt - nrem;
    if (nkept + nnew > TMAX) { C.err |= ST_ECAP_TRI; return; }
    // compact the kept triangles in place (destinations never pass sources)
    int dst = 0;
#pragma unroll
    for (int c = 0; c < TMAX / 32; ++c) {
        if (c >= nchunk) break;
        int t = c * 32 + lane;
        bool keep = t < C.nt && !((outm[c] >> lane) & 1u);
        unsigned km = __ballot_sync(FULL, keep);
        unsigned v = 0;
        double x = 0, y = 0, z = 0;
        if (keep) { v = S.tv[t]; x = S.tx[t]; y = S.ty[t]; z = S.tz[t]; }
        __syncwarp();
        if (keep) {
            int d = dst + __popc(km & lanemask_lt());
            S.tv[d] = v; S.tx[d] = x; S.ty[d] = y; S.tz[d] = z;
        }
        dst += __popc(km);
        __syncwarp();
    }
    // append the new vertices
    for (int e = lane; e < nnew; e += 32) {
        unsigned v = S.stage[e];
        int t = nkept + e;
        S.tv[t] = v;
        double x, y, z;
        plane_vertex(S, v & 255u, (v >> 8) & 255u, kp, x, y, z);
        S.tx[t] = x; S.ty[t] = y; S.tz[t] = z;
    }
    __syncwarp();
    C.nt = nkept + nnew;
    C.np = kp + 1;
    C.cuts++;
    double m = 0.0;
    for (int t = lane; t < C.nt; t += 32) m = fmax(m, S.tx[t] * S.tx[t] + S.ty[t] * S.ty[t] + S.tz[t] * S.tz[t]);
    C.rmax2 = warp_max(m);
}

template <int PREC>
__device__ void flush_batch(ClipSmem &S, int &ncand, CellState &C, int lane)
{
    if (ncand == 0) return;
    sort_candidates(S, ncand, lane);
    for (int k = 0; k < ncand; ++k) {
        if (S.cd[k] > 4.0 * C.rmax2) break;
        clip_by<PREC>(S, k, C, lane);
        if (C.err) break;
    }
    ncand = 0;
    __syncwarp();
}

template <int PREC>
__global__ void __launch_bounds__(32 * CLIP_WARPS)
k_clip(const double4_32a *__restrict__ sorted, const int *__restrict__ start, int64_t n, Grid g, double amin,
       double *__restrict__ vol, double *__restrict__ cen, Slots sl, DevStatus *st, int collect)
{
    __shared__ ClipSmem smem[CLIP_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * CLIP_WARPS + wid;
    if (w >= n) return;
    ClipSmem &S = smem[wid];
    const double4_32a me = sorted[w];
    const double px = me.x, py = me.y, pz = me.z;
    const int self = (int)me.w;
    const double Lx = g.box[0], Ly = g.box[1], Lz = g.box[2];

    // starting box: planes 0..5 = +x,-x,+y,-y,+z,-z self-image bisectors
    if (lane < 6) {
        int d = lane >> 1;
        double sg = (lane & 1) ? -1.0 : 1.0;
        double L = g.box[d];
        S.px[lane] = d == 0 ? sg * L : 0.0;
        S.py[lane] = d == 1 ? sg * L : 0.0;
        S.pz[lane] = d == 2 ? sg * L : 0.0;
        S.po[lane] = 0.5 * L * L;
        S.pnb[lane] = self;
        int s3[3] = {0, 0, 0};
        s3[d] = (lane & 1) ? -1 : 1;
        S.psh[lane] = (s3[0] + 1) + 3 * (s3[1] + 1) + 9 * (s3[2] + 1);
    }
    if (lane < 8) {
        // corner (sx, sy, sz): planes chosen by sign, ordered so det > 0
        int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;  // 1 means negative
        unsigned a = sx, b = 2 + sy, c = 4 + sz;
        // det(sign_x e_x, sign_y e_y, sign_z e_z) = product of signs
        bool neg = (sx ^ sy ^ sz) & 1;
        if (neg) { unsigned t = b; b = c; c = t; }
        S.tv[lane] = a | (b << 8) | (c << 16);
        S.tx[lane] = sx ? -0.5 * Lx : 0.5 * Lx;
        S.ty[lane] = sy ? -0.5 * Ly : 0.5 * Ly;
        S.tz[lane] = sz ? -0.5 * Lz : 0.5 * Lz;
    }
    for (int r = lane; r < PMAX; r += 32) S.bm[r] = 0ull;
    __syncwarp();
    CellState C;
    C.np = 6;
    C.nt = 8;
    C.rmax2 = 0.25 * (Lx * Lx + Ly * Ly + Lz * Lz);
    C.err = 0;
    C.cuts = 0;

    int cb[3];
    {
        double pp[3] = {px, py, pz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int c = (int)floor(pp[d] / g.bs[d]);
            cb[d] = c < 0 ? 0 : (c >= g.g[d] ? g.g[d] - 1 : c);
        }
    }
    int ncand = 0, maxcand = 0;
    int rl = 0, rh = 1;
    bool done = false;
    int rings = 0;
    while (!done && !C.err) {
        const int nb = 2 * rh + 1;
        const int total = nb * nb * nb;
        for (int base = 0; base < total && !C.err; base += 32) {
            int t = base + lane;
            int cur = 0, end = 0;
            int shx = 0, shy = 0, shz = 0;
            if (t < total) {
                int ox = t % nb - rh, oy = (t / nb) % nb - rh, oz = t / (nb * nb) - rh;
                int ch = max(abs(ox), max(abs(oy), abs(oz)));
                if (ch >= rl) {
                    int bx = cb[0] + ox, by = cb[1] + oy, bz = cb[2] + oz;
                    shx = (int)floor((double)bx / g.g[0]);
                    shy = (int)floor((double)by / g.g[1]);
                    shz = (int)floor((double)bz / g.g[2]);
                    bx -= shx * g.g[0];
                    by -= shy * g.g[1];
                    bz -= shz * g.g[2];
                    int b = bx + g.g[0] * (by + g.g[1] * bz);
                    cur = start[b];
                    end = start[b + 1];
                    // images two or more boxes away never cut (positions lie in [0, L))
                    if (abs(shx) > 1 || abs(shy) > 1 || abs(shz) > 1) end = cur;
                }
            }
            const double offx = shx * Lx - px, offy = shy * Ly - py, offz = shz * Lz - pz;
            const int code = (shx + 1) + 3 * (shy + 1) + 9 * (shz + 1);
            const bool selfimg = (abs(shx) + abs(shy) + abs(shz)) <= 1;
            while (__any_sync(FULL, cur < end)) {
                if (ncand + 32 > CBATCH) flush_batch<PREC>(S, ncand, C, lane);
                if (C.err) break;
                bool keep = false;
                double qx = 0, qy = 0, qz = 0, d2 = 0;
                int j = 0;
                if (cur < end) {
                    double4_32a P = sorted[cur];
                    ++cur;
                    j = (int)P.w;
                    qx = P.x + offx; qy = P.y + offy; qz = P.z + offz;
                    d2 = qx * qx + qy * qy + qz * qz;
                    keep = !(j == self && selfimg) && d2 < 4.0 * C.rmax2;
                }
                unsigned km = __ballot_sync(FULL, keep);
                if (keep) {
                    int s = ncand + __popc(km & lanemask_lt());
                    S.cx[s] = qx; S.cy[s] = qy; S.cz[s] = qz; S.cd[s] = d2;
                    S.cid[s] = j; S.csh[s] = code;
                }
                ncand += __popc(km);
                maxcand = max(maxcand, ncand);
                __syncwarp();
            }
        }
        flush_batch<PREC>(S, ncand, C, lane);
        ++rings;
        // radius the gathered rings are guaranteed to cover
        double R = 1e300;
        {
            double pp[3] = {px, py, pz};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double lo = (cb[d] - rh) * g.bs[d], hi = (cb[d] + rh + 1) * g.bs[d];
                R = fmin(R, fmin(pp[d] - lo, hi - pp[d]));
            }
        }
        if (4.0 * C.rmax2 <= R * R) done = true;
        else {
            rl = rh + 1;
            rh = rl;
            if (rh > MAXRING) C.err |= ST_ECAP_RING;
        }
    }

    // ---- finalisation: faces, volume, centroid
    double vl = 0.0, vcx = 0.0, vcy = 0.0, vcz = 0.0;
    if (!C.err) {
        for (int p = lane; p < C.np; p += 32) {
            int t0 = -1;
            unsigned y = 0;
            for (int t = 0; t < C.nt; ++t) {
                unsigned v = S.tv[t];
                unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
                if (a == (unsigned)p) { t0 = t; y = c; break; }
                if (b == (unsigned)p) { t0 = t; y = a; break; }
                if (c == (unsigned)p) { t0 = t; y = b; break; }
            }
            S.fa[p] = 0.0;
            if (t0 < 0) continue;  // plane no longer bounds the cell
            const double qx = S.px[p], qy = S.py[p], qz = S.pz[p];
            const double x0 = S.tx[t0], y0 = S.ty[t0], z0 = S.tz[t0];
            double ax = 0, ay = 0, az = 0;  // previous vertex
            double A2 = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
            int cnt = 1;
            bool ok = false;
            for (int guard = 0; guard < TMAX; ++guard) {
                // next vertex around p: the triangle containing p -> y
                int tn = -1;
                unsigned z = 0;
                for (int t = 0; t < C.nt; ++t) {
                    unsigned v = S.tv[t];
                    unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
                    if (a == (unsigned)p && b == y) { tn = t; z = c; break; }
                    if (b == (unsigned)p && c == y) { tn = t; z = a; break; }
                    if (c == (unsigned)p && a == y) { tn = t; z = b; break; }
                }
                if (tn < 0) break;
                if (tn == t0) { ok = true; break; }
                const double bx = S.tx[tn], by = S.ty[tn], bz = S.tz[tn];
                if (cnt >= 2) {
                    const double ux = ax - x0, uy = ay - y0, uz = az - z0;
                    const double vx = bx - x0, vy = by - y0, vz = bz - z0;
                    const double w = qx * (uy * vz - uz * vy) + qy * (uz * vx - ux * vz) + qz * (ux * vy - uy * vx);
                    A2 += w;
                    sx += w * (x0 + ax + bx);
                    sy += w * (y0 + ay + by);
                    sz += w * (z0 + az + bz);
                }
                ax = bx; ay = by; az = bz;
                ++cnt;
                y = z;
            }
            if (!ok) { C.err |= ST_EDEGEN; continue; }
            const double ql = sqrt(qx * qx + qy * qy + qz * qz);
            const double area = 0.5 * fabs(A2) / ql;
            const double fx = A2 != 0.0 ? sx / (3.0 * A2) : x0;
            const double fy = A2 != 0.0 ? sy / (3.0 * A2) : y0;
            const double fz = A2 != 0.0 ? sz / (3.0 * A2) : z0;
            S.fa[p] = area;
            S.fcx[p] = fx; S.fcy[p] = fy; S.fcz[p] = fz;
            const double vp = area * ql / 6.0;  // A h / 3 with h = |q| / 2
            vl += vp;
            vcx += 0.75 * vp * fx;
            vcy += 0.75 * vp * fy;
            vcz += 0.75 * vp * fz;
        }
        C.err = __reduce_or_sync(FULL, (unsigned)C.err);
    }
    __syncwarp();
    vl = warp_sum(vl);
    vcx = warp_sum(vcx);
    vcy = warp_sum(vcy);
    vcz = warp_sum(vcz);

    int nface = 0;
    if (!C.err) {
        const int64_t sbase = (int64_t)self * MAXF;
        for (int p0 = 0; p0 < C.np; p0 += 32) {
            int p = p0 + lane;
            bool keep = p < C.np && S.fa[p] > amin;
            unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                int k = nface + __popc(km & lanemask_lt());
                if (k < MAXF) {
                    int64_t s = sbase + k;
                    sl.nb[s] = S.pnb[p];
                    sl.sh[s] = (unsigned char)S.psh[p];
                    sl.area[s] = S.fa[p];
                    const int64_t ns = n * (int64_t)MAXF;
                    sl.fc[s] = px + S.fcx[p];
                    sl.fc[ns + s] = py + S.fcy[p];
                    sl.fc[2 * ns + s] = pz + S.fcz[p];
                }
            }
            nface += __popc(km);
        }
        if (nface > MAXF) C.err |= ST_ECAP_FACE;
    }
    if (lane == 0) {
        if (C.err) {
            atomicOr(&st->flags, C.err);
            atomicExch(&st->bad_cell, self);
            nface = 0;
        }
        sl.cnt[self] = nface;
        vol[self] = vl;
        cen[self] = px + vcx / vl;
        cen[n + self] = py + vcy / vl;
        cen[2 * n + self] = pz + vcz / vl;
        if (collect) {
            atomicMax(&st->max_cand, maxcand);
            atomicMax(&st->max_planes, C.np);
            atomicMax(&st->max_tris, C.nt);
            if (rings > 1) atomicAdd(&st->multi_ring, 1);
            atomicAdd(&st->cuts, (unsigned long long)C.cuts);
        }
    }
}

void launch_clip(const double4_32a *sorted, const int *start, int64_t n, const Grid &g, double amin, int precision,
                 double *vol, double *cen, Slots sl, DevStatus *st, cudaStream_t s)
{
    int64_t nb = (n + CLIP_WARPS - 1) / CLIP_WARPS;
    if (precision == 0)
        k_clip<0><<<(unsigned)nb, 32 * CLIP_WARPS, 0, s>>>(sorted, start, n, g, amin, vol, cen, sl, st, 1);
    else
        k_clip<1><<<(unsigned)nb, 32 * CLIP_WARPS, 0, s>>>(sorted, start, n, g, amin, vol, cen, sl, st, 1);
}

}  // namespace mm
