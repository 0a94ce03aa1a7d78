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
//    intersection of those three planes.  A cut removes the triangles beyond
//    the plane; the directed edges of removed triangles whose reverse edge is
//    not also removed form the rim of the hole, and each rim edge x->y
//    becomes a new triangle (x, y, k).  A 64x64 bit matrix in shared memory
//    answers "is y->x removed" in O(1); it is marked with 32-bit atomics.
//  * Candidates come from a uniform grid of bins, ring by ring (Chebyshev
//    distance in bins), filtered by |q| < 2 r_max, sorted by (|q|, id, image)
//    with a warp bitonic sort, and clipped in that order.  The cell is
//    complete once 2 r_max is inside the radius the gathered rings cover.
//  * Geometry: a face's polygon is walked around its plane in the dual, its
//    area and centroid come from a fan about its first vertex, and the cell
//    volume and centroid from the pyramids (apex p)
//    over the faces: V_f = A h / 3 with h = |q|/2, centroid 3/4 of the way
//    from p to the face centroid.
//
// Precision.  GB300 issues FP64 at 1/64 of the FP32 rate, and the warp-wide
// FP64 instruction count bounds this kernel.  PREC 0 (clip_filter = 0) solves
// every vertex in FP64 when it is created and classifies it in FP64.  PREC 1
// (clip_filter = 1, the default) keeps the
// vertices in FP32 during clipping together with a forward error bound, and
// classifies with FP32 where the bound settles the sign; where it does not,
// it solves that vertex in FP64 and classifies exactly as PREC 0 does.  At the
// end every vertex is solved in FP64 from its three planes.  Both variants
// therefore take the same decisions and produce the same FP64 geometry.
// Ties: a vertex lies beyond a plane only past a margin of 2^-40..2^-39 of the
// plane's offset, so vertices on it (co-spherical generators of exact
// lattices, where one point has several representations with different
// rounding) are kept consistently.
#include "mm_internal.cuh"

namespace mm {

constexpr unsigned FULL = 0xffffffffu;
#ifndef MM_CLIP_MAXNREG
#define MM_CLIP_MAXNREG 128  // registers per thread of the clipping kernel
#endif
constexpr int CBATCH = 64;  // candidate buffer; flushed (sorted + clipped) when full

// Per-cell capacities of one instance of the clipper: planes, vertices, new
// vertices per cut, faces written, search rings and edge-table slots.  The
// main instance runs every cell; the large one re-clips the cells that
// overflowed the main one's lists.
template <int PM_, int TM_, int NS_, int MF_, int MR_, int ETAB_, bool BIG_>
struct Caps {
    static constexpr int PM = PM_, TM = TM_, NS = NS_, MF = MF_, MR = MR_, ETAB = ETAB_;
    static constexpr bool BIG = BIG_;
    static constexpr int BMW = PM_ / 32;                  // bit-matrix words per plane row
    static constexpr int PB = PM_ == 64 ? 6 : 7;          // bits of a plane index (edge-table keys)
    static constexpr int TB = TM_ == 128 ? 7 : 8;         // bits of a triangle index (edge-table entries)
    static constexpr int EH = ETAB_ == 256 ? 24 : 22;     // hash shift, 32 - log2(ETAB)
    static constexpr int CID = PM_ > CBATCH ? PM_ : CBATCH;  // candidate ids, reused as first[plane]
};
using CapMain = Caps<PMAX, TMAX, NSTAGE, MAXF, MAXRING, 256, false>;
using CapBig = Caps<PMAX_BIG, TMAX_BIG, NSTAGE_BIG, MAXF_BIG, MAXRING_BIG, 1024, true>;
static_assert(CBATCH <= PMAX, "the candidate buffer shares its storage with the per-face arrays");
static_assert(3 * TMAX_BIG <= 1024 * 3 / 4, "the large edge table holds every corner");

// Vertex storage.  PREC 0 keeps FP64 vertices throughout.  PREC 1 keeps FP32
// vertices with their error bounds while clipping and solves the FP64
// vertices only at the end, when the FP32 copies and |v|^2 bounds are dead:
// the two sets share the same bytes.
template <int PREC, class CAP>
struct VertStore;
template <class CAP>
struct VertStore<0, CAP> {
    double tx[CAP::TM], ty[CAP::TM], tz[CAP::TM];
    long long tr2[CAP::TM];  // bits of |v|^2
    float4 tf[1];
};
template <class CAP>
struct VertStore<1, CAP> {
    union {
        struct {
            double tx[CAP::TM], ty[CAP::TM], tz[CAP::TM];  // after clipping
        };
        struct {
            long long tr2[CAP::TM];  // bits of an FP32 upper bound of |v|^2
            float4 tf[CAP::TM];      // FP32 vertex (x, y, z) and its error bound (w)
        };
    };
};

template <int PREC, class CAP>
struct ClipSmem : VertStore<PREC, CAP> {
    union {
        struct {
            double x[CBATCH], y[CBATCH], z[CBATCH];
            long long d2[CBATCH];  // bit pattern of |q|^2 (non-negative: orders like the value)
            float4 cf[CBATCH];     // FP32 copies (q, |q|^2 / 2) for filtered clipping
        } c;
        struct {
            double a[CAP::PM], x[CAP::PM], y[CAP::PM], z[CAP::PM];  // per-face area and centroid
            unsigned etab[CAP::ETAB];                               // directed edge -> (triangle, third corner)
        } f;
    } u;
    int cid[CAP::CID], csh[CBATCH];
    unsigned char perm[CBATCH];  // clipping order of the buffered candidates
    double px[CAP::PM], py[CAP::PM], pz[CAP::PM], po[CAP::PM];  // planes x.q <= po
    int pnb[CAP::PM], psh[CAP::PM];
    unsigned tv[CAP::TM];                  // a | b << 8 | c << 16
    unsigned bm[CAP::BMW * CAP::PM];       // removed directed edges x -> y: bit y % 32 of word BMW x + y / 32
    unsigned stage[CAP::NS];               // triangles created by the current cut
    double off[9];               // image offsets s L - p: off[3 d + s + 1], s = -1, 0, +1
    float offf[9];               // their FP32 roundings (the gather filter)
    float4 pf[PREC ? CAP::PM : 1];  // FP32 planes (q, o)
    float pfn[PREC ? CAP::PM : 1];  // FP32 |q| = sqrt(2 o) of each plane (for the vertex error bound)
};

// Sets of plane indices (one bit per plane slot) for the rim check and the
// slot recycling: one 64-bit word for the main instance, two for the large.
template <int PM>
struct PMask;
template <>
struct PMask<64> {
    unsigned long long w = 0ull;
    __device__ __forceinline__ void set(unsigned b) { w |= 1ull << b; }
    __device__ __forceinline__ int popc() const { return __popcll(w); }
    __device__ __forceinline__ bool operator!=(const PMask &o) const { return w != o.w; }
};
template <>
struct PMask<128> {
    unsigned long long w = 0ull, h = 0ull;
    __device__ __forceinline__ void set(unsigned b)
    {
        if (b < 64u) w |= 1ull << b;
        else h |= 1ull << (b - 64u);
    }
    __device__ __forceinline__ int popc() const { return __popcll(w) + __popcll(h); }
    __device__ __forceinline__ bool operator!=(const PMask &o) const { return w != o.w || h != o.h; }
};

// Rarely taken integer work of the gather, kept out of line so that the hot
// loop around it stays small (the kernel is sensitive to instruction-cache
// misses): floor(a / b) for b > 0 (images beyond the neighbouring boxes), and
// the bin offsets of entry t of ring block rh of side nb = 2 rh + 1 (rings 3
// and beyond).
__device__ __noinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __noinline__ int3 ring_offset(int t, int nb, int rh)
{
    return make_int3(t % nb - rh, (t / nb) % nb - rh, t / (nb * nb) - rh);
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// Warp-wide sums of four values, on every lane, in a fixed order.  Each
// exchange halves the number of partial sums a lane keeps (lanes with bit 4
// clear keep a and b, the others c and d; then bit 3 splits those), so a
// lane does six FP64 additions instead of twenty.
__device__ __forceinline__ void warp_sum4(double &a, double &b, double &c, double &d, int lane)
{
    const bool h4 = (lane & 16) != 0;
    double k0 = h4 ? c : a, k1 = h4 ? d : b;
    const double s0 = h4 ? a : c, s1 = h4 ? b : d;
    k0 += __shfl_xor_sync(FULL, s0, 16);
    k1 += __shfl_xor_sync(FULL, s1, 16);
    const bool h3 = (lane & 8) != 0;
    double k = h3 ? k1 : k0;
    k += __shfl_xor_sync(FULL, h3 ? k0 : k1, 8);
    k += __shfl_xor_sync(FULL, k, 4);
    k += __shfl_xor_sync(FULL, k, 2);
    k += __shfl_xor_sync(FULL, k, 1);
    // lanes 0-7 hold the sum of a, 8-15 of b, 16-23 of c, 24-31 of d
    a = __shfl_sync(FULL, k, 0);
    b = __shfl_sync(FULL, k, 8);
    c = __shfl_sync(FULL, k, 16);
    d = __shfl_sync(FULL, k, 24);
}

// Bit pattern of (double) f for a finite f >= 0: a normal float's exponent
// moved to the double bias (integer operations), else the conversion.
__device__ __forceinline__ long long dbits_of_float(float f)
{
    const unsigned fb = __float_as_uint(f);
    const unsigned e = fb >> 23;
    if (e != 0u && e < 255u)
        return (long long)(((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)(fb & 0x7fffffu) << 29));
    return __double_as_longlong((double)f);
}

// Magnitude order of doubles by their bit patterns (non-negative values, or
// absolute values): an integer comparison in place of an FP64 one.
__device__ __forceinline__ long long abs_bits(double x)
{
    return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}
// Warp-wide maximum of a non-negative 64-bit value: the high words first,
// then the low words of the lanes holding the largest high word.
__device__ __forceinline__ long long warp_max_nonneg(long long v)
{
    const unsigned long long u = (unsigned long long)v;
    const unsigned hi = __reduce_max_sync(FULL, (unsigned)(u >> 32));
    const unsigned lo = __reduce_max_sync(FULL, (unsigned)(u >> 32) == hi ? (unsigned)u : 0u);
    return (long long)(((unsigned long long)hi << 32) | lo);
}
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v)
{
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)v);
    const unsigned hi = __reduce_or_sync(FULL, (unsigned)(v >> 32));
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ PMask<64> warp_or(PMask<64> m)
{
    m.w = warp_or64(m.w);
    return m;
}
__device__ __forceinline__ PMask<128> warp_or(PMask<128> m)
{
    m.w = warp_or64(m.w);
    m.h = warp_or64(m.h);
    return m;
}
// The lowest plane slot below np that no vertex refers to, or -1.
__device__ __forceinline__ int first_free(const PMask<64> &live, int np)
{
    const unsigned long long used = np >= 64 ? ~0ull : ((1ull << np) - 1ull);
    const unsigned long long freeb = used & ~live.w;
    return freeb ? __ffsll((long long)freeb) - 1 : -1;
}
__device__ __forceinline__ int first_free(const PMask<128> &live, int np)
{
    const unsigned long long u0 = np >= 64 ? ~0ull : ((1ull << np) - 1ull);
    const unsigned long long u1 = np >= 128 ? ~0ull : (np <= 64 ? 0ull : ((1ull << (np - 64)) - 1ull));
    const unsigned long long f0 = u0 & ~live.w, f1 = u1 & ~live.h;
    if (f0) return __ffsll((long long)f0) - 1;
    return f1 ? 64 + __ffsll((long long)f1) - 1 : -1;
}

// Intersection of planes a, b, c in FP64 with explicitly rounded operations
// (so every caller gets the same bits):
// x = (o_a (q_b x q_c) + o_b (q_c x q_a) + o_c (q_a x q_b)) / det(q_a, q_b, q_c).
template <class S_t>
__device__ __forceinline__ void vertex64(const S_t &S, int a, int b, int c, double &x, double &y, double &z)
{
    const double ax = S.px[a], ay = S.py[a], az = S.pz[a], ao = S.po[a];
    const double bx = S.px[b], by = S.py[b], bz = S.pz[b], bo = S.po[b];
    const double cx = S.px[c], cy = S.py[c], cz = S.pz[c], co = S.po[c];
    const double bcx = __fma_rn(by, cz, -__dmul_rn(bz, cy)), bcy = __fma_rn(bz, cx, -__dmul_rn(bx, cz)),
                 bcz = __fma_rn(bx, cy, -__dmul_rn(by, cx));
    const double cax = __fma_rn(cy, az, -__dmul_rn(cz, ay)), cay = __fma_rn(cz, ax, -__dmul_rn(cx, az)),
                 caz = __fma_rn(cx, ay, -__dmul_rn(cy, ax));
    const double abx = __fma_rn(ay, bz, -__dmul_rn(az, by)), aby = __fma_rn(az, bx, -__dmul_rn(ax, bz)),
                 abz = __fma_rn(ax, by, -__dmul_rn(ay, bx));
    const double det = __fma_rn(ax, bcx, __fma_rn(ay, bcy, __dmul_rn(az, bcz)));
    const double inv = __drcp_rn(det);
    x = __dmul_rn(__fma_rn(ao, bcx, __fma_rn(bo, cax, __dmul_rn(co, abx))), inv);
    y = __dmul_rn(__fma_rn(ao, bcy, __fma_rn(bo, cay, __dmul_rn(co, aby))), inv);
    z = __dmul_rn(__fma_rn(ao, bcz, __fma_rn(bo, caz, __dmul_rn(co, abz))), inv);
}

// The exact-path predicate: is vertex v strictly beyond the plane x.q <= off?
__device__ __forceinline__ bool beyond64(double qx, double qy, double qz, double off, double x, double y, double z)
{
    return __fma_rn(qx, x, __fma_rn(qy, y, __dmul_rn(qz, z))) > off;
}

// |q|^2 / 2 from the bit pattern of |q|^2: halving a normal double lowers its
// exponent by one, an integer operation.
__device__ __forceinline__ double half_of(long long d2bits)
{
    if (((d2bits >> 52) & 0x7ff) > 1) return __longlong_as_double(d2bits - (1LL << 52));
    return 0.5 * __longlong_as_double(d2bits);
}

__device__ __forceinline__ long long r2_bits64(double x, double y, double z)
{
    return __double_as_longlong(__fma_rn(x, x, __fma_rn(y, y, __dmul_rn(z, z))));
}

// Intersection of planes a, b, c in FP32 with a bound on its distance to the
// exact intersection.  With P = |q_a||q_b||q_c|, H = P / |det| >= 1 and
// u = 2^-24, first-order rounding analysis of Cramer's rule (inputs rounded
// to FP32, cross products, determinant, numerator, scaling) gives
// |v~ - v| <= u H (5.5 sum|q| + 13 |v|); the bound used is three times that.
// Ill-conditioned intersections get an infinite bound (always checked in FP64).
template <class S_t>
__device__ __forceinline__ void vertex32(const S_t &S, int a, int b, int c, float &x, float &y, float &z,
                                         float &err)
{
    const float4 Pa = S.pf[a], Pb = S.pf[b], Pc = S.pf[c];
    const float ax = Pa.x, ay = Pa.y, az = Pa.z, ao = Pa.w;
    const float bx = Pb.x, by = Pb.y, bz = Pb.z, bo = Pb.w;
    const float cx = Pc.x, cy = Pc.y, cz = Pc.z, co = Pc.w;
    const float bcx = fmaf(by, cz, -bz * cy), bcy = fmaf(bz, cx, -bx * cz), bcz = fmaf(bx, cy, -by * cx);
    const float cax = fmaf(cy, az, -cz * ay), cay = fmaf(cz, ax, -cx * az), caz = fmaf(cx, ay, -cy * ax);
    const float abx = fmaf(ay, bz, -az * by), aby = fmaf(az, bx, -ax * bz), abz = fmaf(ax, by, -ay * bx);
    const float det = fmaf(ax, bcx, fmaf(ay, bcy, az * bcz));
    const float inv = __frcp_rn(det);
    x = fmaf(ao, bcx, fmaf(bo, cax, co * abx)) * inv;
    y = fmaf(ao, bcy, fmaf(bo, cay, co * aby)) * inv;
    z = fmaf(ao, bcz, fmaf(bo, caz, co * abz)) * inv;
    // |q_k| = sqrt(2 o_k)
    const float la = S.pfn[a], lb = S.pfn[b], lc = S.pfn[c];
    const float H = la * lb * lc * fabsf(inv);  // P / |det| through the reciprocal (the factor 3 covers its ulp)
    const float vn = fabsf(x) + fabsf(y) + fabsf(z);
    const float u = 5.9604645e-8f;
    err = 3.0f * u * H * (5.5f * (la + lb + lc) + 13.0f * vn);
    // The analysis assumes no FP32 underflow or overflow: the numerators grow
    // like |q|^4 and the determinant like |q|^3, so planes much nearer than
    // 2^-28 or farther than 2^28 (tiny or huge boxes) are solved exactly.
    const float qlo = fminf(la, fminf(lb, lc)), qhi = fmaxf(la, fmaxf(lb, lc));
    if (!(u * H < 1e-3f) || !(err < 1e30f) || !(qlo >= 3.7252903e-9f) || !(qhi <= 268435456.0f))
        err = __int_as_float(0x7f800000);  // +inf
}

// The rare exact paths of the filtered clipper, kept out of line so that the
// unrolled loops around them stay small: the FP64 plane test of a vertex the
// FP32 bound cannot settle, and the FP64 solve of an ill-conditioned vertex.
template <class S_t>
__device__ __noinline__ bool beyond_exact(const S_t &S, unsigned v, double qx, double qy, double qz, double off)
{
    double x, y, z;
    vertex64(S, v & 255u, (v >> 8) & 255u, (v >> 16) & 255u, x, y, z);
    return beyond64(qx, qy, qz, off, x, y, z);
}
template <class S_t>
__device__ __noinline__ void vertex64_call(const S_t &S, int a, int b, int c, double &x, double &y, double &z)
{
    vertex64(S, a, b, c, x, y, z);
}

// Face walk without the edge table (cells of more than 64 vertices): the
// first triangle holding plane p (and the corner before p in it), and the
// triangle holding the directed edge p -> y (and its third corner), by scans.
__device__ __noinline__ int scan_first(const unsigned *tv, int nt, unsigned p, unsigned &y)
{
    for (int t = 0; t < nt; ++t) {
        const unsigned v = tv[t];
        const unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
        if (a == p) { y = c; return t; }
        if (b == p) { y = a; return t; }
        if (c == p) { y = b; return t; }
    }
    return -1;
}
__device__ __noinline__ int scan_next(const unsigned *tv, int nt, unsigned p, unsigned y, unsigned &z)
{
    for (int t = 0; t < nt; ++t) {
        const unsigned v = tv[t];
        const unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
        if (a == p && b == y) { z = c; return t; }
        if (b == p && c == y) { z = a; return t; }
        if (c == p && a == y) { z = b; return t; }
    }
    return -1;
}

// Candidate order: (|q|^2, id, image code).
template <class S_t>
__device__ __forceinline__ bool cand_less(const S_t &S, int a, int b)
{
    if (S.u.c.d2[a] != S.u.c.d2[b]) return S.u.c.d2[a] < S.u.c.d2[b];
    if (S.cid[a] != S.cid[b]) return S.cid[a] < S.cid[b];
    return S.csh[a] < S.csh[b];
}

template <class S_t>
__device__ __forceinline__ void cand_swap(S_t &S, int a, int b)
{
    double t;
    t = S.u.c.x[a]; S.u.c.x[a] = S.u.c.x[b]; S.u.c.x[b] = t;
    t = S.u.c.y[a]; S.u.c.y[a] = S.u.c.y[b]; S.u.c.y[b] = t;
    t = S.u.c.z[a]; S.u.c.z[a] = S.u.c.z[b]; S.u.c.z[b] = t;
    long long l = S.u.c.d2[a]; S.u.c.d2[a] = S.u.c.d2[b]; S.u.c.d2[b] = l;
    int v;
    v = S.cid[a]; S.cid[a] = S.cid[b]; S.cid[b] = v;
    v = S.csh[a]; S.csh[a] = S.csh[b]; S.csh[b] = v;
}

// Warp bitonic sort of the first m candidates (padded to a power of two).
template <class S_t>
__device__ void sort_candidates(S_t &S, int m, int lane)
{
    int P = 1;
    while (P < m) P <<= 1;
    for (int t = m + lane; t < P; t += 32) {
        S.u.c.d2[t] = 0x7fffffffffffffffLL;
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
    long long lim;  // bits of 4 r_max^2: a candidate with |q|^2 above it cannot cut
    float limk;     // FP32 gather threshold: at least lim plus the FP32 rounding of |q|^2
    float slack;    // 2e-6 max(L): the position-rounding term of that margin
    int err;
    int cuts;
    bool strict;     // tie rule: strict (q.v > o) instead of the margin (retry of an inconsistent cut)
    // work counters (warp-uniform), reported when the caller collects stats
    unsigned pred64, solve64, fan64, tested;
};

// The security limit from each lane's largest |v|^2 bound over the vertices
// it handled (the kept ones it compacted and the new ones it solved).
template <int PREC>
__device__ __forceinline__ void update_limit(CellState &C, long long m)
{
    float m4;
    if constexpr (PREC == 0) {
        m = warp_max_nonneg(m);
        C.lim = __double_as_longlong(4.0 * __longlong_as_double(m));
        m4 = (float)__longlong_as_double(C.lim);
    } else {
        // the bounds are positive floats: their bit patterns fit 32 bits, and
        // 4 (double) f is f's exponent moved to the double bias plus two
        const unsigned fb = __reduce_max_sync(FULL, (unsigned)m);
        const unsigned e = fb >> 23;
        if (e != 0u && e < 255u)
            C.lim = (long long)(((unsigned long long)(e + (1023u - 127u + 2u)) << 52) |
                                ((unsigned long long)(fb & 0x7fffffu) << 29));
        else
            C.lim = __double_as_longlong(4.0 * (double)__int_as_float((int)fb));
        m4 = 4.0f * __int_as_float((int)fb);
    }
    // An FP32 |q|^2 from FP32 copies of positions and offsets is within
    // 2e-7 |q|^2 + 1.3e-6 max(L) |q| of the exact one (positions and offsets
    // below 3 max(L)): this threshold keeps every candidate the exact test would.
    C.limk = fmaf(m4, 1.00001f, C.slack * sqrtf(m4));
}

// Clip the cell by candidate k.  Warp-uniform control flow throughout.
// The removed-vertex masks of a cut, one 32-bit ballot per chunk of 32
// vertices, held in two 64-bit registers: the chunk loops then need no
// unrolling to keep them out of local memory (a smaller kernel body).
template <int TM>
struct ChunkMask;
template <>
struct ChunkMask<128> {
    unsigned long long lo = 0ull, hi = 0ull;
    __device__ __forceinline__ unsigned get(int c) const
    {
        return (unsigned)((c < 2 ? lo : hi) >> (32 * (c & 1)));
    }
    __device__ __forceinline__ void put(int c, unsigned m)
    {
        const unsigned long long v = (unsigned long long)m << (32 * (c & 1));
        if (c < 2) lo |= v;
        else hi |= v;
    }
    __device__ __forceinline__ bool any() const { return (lo | hi) != 0ull; }
    __device__ __forceinline__ int count() const { return __popcll(lo) + __popcll(hi); }
};
template <>
struct ChunkMask<256> {
    unsigned long long w0 = 0ull, w1 = 0ull, w2 = 0ull, w3 = 0ull;
    __device__ __forceinline__ unsigned get(int c) const
    {
        const unsigned long long w = c < 2 ? w0 : (c < 4 ? w1 : (c < 6 ? w2 : w3));
        return (unsigned)(w >> (32 * (c & 1)));
    }
    __device__ __forceinline__ void put(int c, unsigned m)
    {
        const unsigned long long v = (unsigned long long)m << (32 * (c & 1));
        if (c < 2) w0 |= v;
        else if (c < 4) w1 |= v;
        else if (c < 6) w2 |= v;
        else w3 |= v;
    }
    __device__ __forceinline__ bool any() const { return (w0 | w1 | w2 | w3) != 0ull; }
    __device__ __forceinline__ int count() const { return __popcll(w0) + __popcll(w1) + __popcll(w2) + __popcll(w3); }
};

// A new vertex of the cut by plane kp: the intersection of the rim edge's two
// planes with kp, FP64 (PREC 0) or FP32 with its error bound (PREC 1), and the
// bits of (a bound of) |v|^2.
template <int PREC, class S_t>
__device__ __forceinline__ void new_vertex(const S_t &S, unsigned nvt, int kp, long long &nr2, double &nX, double &nY,
                                           double &nZ, float4 &nf)
{
    if constexpr (PREC == 0) {
        vertex64(S, nvt & 255u, (nvt >> 8) & 255u, kp, nX, nY, nZ);
        nr2 = r2_bits64(nX, nY, nZ);
    } else {
        float x, y, z, er;
        vertex32(S, nvt & 255u, (nvt >> 8) & 255u, kp, x, y, z, er);
        if (!(er < 1e30f)) {
            // ill-conditioned intersection: solve it in FP64 now and keep
            // its FP32 rounding, whose error is then one rounding per axis
            double X, Y, Z;
            vertex64_call(S, nvt & 255u, (nvt >> 8) & 255u, kp, X, Y, Z);
            x = (float)X; y = (float)Y; z = (float)Z;
            er = 1.2e-7f * (fabsf(x) + fabsf(y) + fabsf(z)) + 1e-38f;
        }
        nf = make_float4(x, y, z, er);
        // an FP32 upper bound of (|v| + er)^2 <= |v|^2 + er (2 |v|_1 + er),
        // kept as the bit pattern of a positive float
        const float s2 = fmaf(x, x, fmaf(y, y, z * z));
        const float l1 = fabsf(x) + fabsf(y) + fabsf(z);
        nr2 = (long long)__float_as_int(fmaf(er, fmaf(2.0f, l1, er), s2) * 1.00001f);
    }
}

template <int PREC, class CAP>
__device__ void clip_by(ClipSmem<PREC, CAP> &S, int k, CellState &C, int lane)
{
    constexpr int BMW = CAP::BMW;
    const double qx = S.u.c.x[k], qy = S.u.c.y[k], qz = S.u.c.z[k];
    const double off = half_of(S.u.c.d2[k]);
    // A vertex is beyond the plane when q.v exceeds the offset by a margin of
    // 2^-40..2^-39 of it (2^13 units in the last place, an integer add on the
    // bit pattern): a vertex exactly on the plane (co-spherical generators,
    // exact lattices) stays, whatever rounding its several representations
    // carry, so copies of one point are never split across the plane.  The
    // planes themselves, and every vertex solved from them, are exact.  The
    // margin can itself split distinct points that lie within it of a plane
    // (lattices perturbed by about 1e-12..1e-9 of a spacing); a cell whose cut
    // is then inconsistent is clipped again with the strict rule (C.strict),
    // which decides those by the geometry.
    const double offk = C.strict ? off : __longlong_as_double(__double_as_longlong(off) + (1LL << 13));
    const int nchunk = (C.nt + 31) >> 5;
    ChunkMask<CAP::TM> outm;
    C.tested++;
    if (PREC == 0) C.pred64 += C.nt;
    float fqx = 0.f, fqy = 0.f, fqz = 0.f, foff = 0.f, fqn = 0.f;
    if constexpr (PREC == 1) {
        const float4 F = S.u.c.cf[k];
        fqx = F.x; fqy = F.y; fqz = F.z; foff = F.w;
        fqn = sqrtf(2.0f * foff) * 1.0000005f;
    }
#pragma unroll 1
    for (int c = 0; c < nchunk; ++c) {
        bool o = false;
        const int t = c * 32 + lane;
        const bool live = t < C.nt;
        if constexpr (PREC == 0) {
            if (live) o = beyond64(qx, qy, qz, offk, S.tx[t], S.ty[t], S.tz[t]);
        } else {
            bool unsure = false;
            if (live) {
                const float4 V = S.tf[t];
                const float vx = V.x, vy = V.y, vz = V.z;
                const float s = fmaf(fqx, vx, fmaf(fqy, vy, fmaf(fqz, vz, -foff)));
                const float mag = fabsf(fqx * vx) + fabsf(fqy * vy) + fabsf(fqz * vz) + foff;
                const float B = fqn * V.w + 16.0f * 5.9604645e-8f * mag;
                // the margin is below 2^-19 B, so B (1 + 1e-5) still settles the sign
                if (s > B * 1.00001f) o = true;
                else if (s < -B) o = false;
                else unsure = true;
            }
            const unsigned um = __ballot_sync(FULL, unsure);
            if (um) {
                C.pred64 += __popc(um);
                C.solve64 += __popc(um);
                if (unsure) o = beyond_exact(S, S.tv[t], qx, qy, qz, offk);
            }
        }
        outm.put(c, __ballot_sync(FULL, o));
        if (o) {
            // mark the directed edges of the removed triangle
            const unsigned v = S.tv[t];
            const unsigned a = v & 255u, b = (v >> 8) & 255u, cc = (v >> 16) & 255u;
            atomicOr(&S.bm[BMW * a + (b >> 5)], 1u << (b & 31u));
            atomicOr(&S.bm[BMW * b + (cc >> 5)], 1u << (cc & 31u));
            atomicOr(&S.bm[BMW * cc + (a >> 5)], 1u << (a & 31u));
        }
    }
    if (!outm.any()) return;
    // the new plane takes a fresh slot while fewer than 32 are in use (one
    // lane per face when the faces are summed); beyond that, the lowest slot
    // no vertex refers to (a face that has vanished frees its slot), else a
    // fresh one: PMAX bounds the live faces
    int kp;
    if (C.np < 32) {
        kp = C.np;
    } else {
        PMask<CAP::PM> live;
        for (int t = lane; t < C.nt; t += 32) {
            const unsigned v = S.tv[t];
            live.set(v & 255u);
            live.set((v >> 8) & 255u);
            live.set((v >> 16) & 255u);
        }
        live = warp_or(live);
        kp = first_free(live, C.np);
        if (kp < 0) {
            if (C.np >= CAP::PM) { C.err |= ST_ECAP_PLANE; return; }
            kp = C.np;
        }
    }
    if (lane == 0) {
        S.px[kp] = qx; S.py[kp] = qy; S.pz[kp] = qz; S.po[kp] = off;
        S.pnb[kp] = S.cid[k]; S.psh[kp] = S.csh[k];
        if constexpr (PREC == 1) {
            S.pf[kp] = make_float4(fqx, fqy, fqz, foff);
            S.pfn[kp] = sqrtf(2.0f * foff);
        }
    }
    __syncwarp();
    // rim edges: removed x->y whose reverse y->x is not removed
    int nnew = 0;
    PMask<CAP::PM> xs, ys;
#pragma unroll 1
    for (int c = 0; c < nchunk; ++c) {
        const unsigned oc = outm.get(c);
        if (oc == 0) continue;  // warp-uniform
        // rim edges of this lane's removed triangle, kept in registers
        unsigned e0 = 0, e1 = 0, e2 = 0;
        bool f0 = false, f1 = false, f2 = false;
        if ((oc >> lane) & 1u) {
            const unsigned v = S.tv[c * 32 + lane];
            const unsigned a = v & 255u, b = (v >> 8) & 255u, cc = (v >> 16) & 255u;
            const unsigned hk = (unsigned)kp << 16;
            f0 = !((S.bm[BMW * b + (a >> 5)] >> (a & 31u)) & 1u);    // a -> b
            f1 = !((S.bm[BMW * cc + (b >> 5)] >> (b & 31u)) & 1u);   // b -> cc
            f2 = !((S.bm[BMW * a + (cc >> 5)] >> (cc & 31u)) & 1u);  // cc -> a
            e0 = a | (b << 8) | hk;
            e1 = b | (cc << 8) | hk;
            e2 = cc | (a << 8) | hk;
            if (f0) { xs.set(a); ys.set(b); }
            if (f1) { xs.set(b); ys.set(cc); }
            if (f2) { xs.set(cc); ys.set(a); }
        }
        const int cnt = (int)f0 + (int)f1 + (int)f2;
        // exclusive prefix of cnt (0..3) from the ballots of its two bits
        const unsigned b0 = __ballot_sync(FULL, cnt & 1), b1 = __ballot_sync(FULL, cnt & 2);
        const unsigned lt = lanemask_lt();
        const int tot = __popc(b0) + 2 * __popc(b1);
        int o = nnew + __popc(b0 & lt) + 2 * __popc(b1 & lt);
        if (f0) { if (o < CAP::NS) S.stage[o] = e0; ++o; }
        if (f1) { if (o < CAP::NS) S.stage[o] = e1; ++o; }
        if (f2) { if (o < CAP::NS) S.stage[o] = e2; ++o; }
        nnew += tot;
    }
    __syncwarp();
    for (int r = lane; r < BMW * C.np; r += 32) S.bm[r] = 0u;
    xs = warp_or(xs);
    ys = warp_or(ys);
    if (nnew > CAP::NS) { C.err |= ST_ECAP_STAGE; return; }
    if (nnew < 3 || xs != ys || xs.popc() != nnew) { C.err |= ST_EDEGEN_CUT; return; }
    const int nrem = outm.count();
    const int nkept = C.nt - nrem;
    if (nkept + nnew > CAP::TM) { C.err |= ST_ECAP_TRI; return; }
    // the new vertices first, one per lane (nnew <= 32), kept in registers:
    // their arithmetic then overlaps the compaction's shared-memory traffic
    long long mr = 0;  // this lane's largest |v|^2 bound, for the new limit
    const bool mk = lane < nnew;
    unsigned nvt = 0;
    long long nr2 = 0;
    double nX = 0.0, nY = 0.0, nZ = 0.0;
    float4 nf = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mk) {
        nvt = S.stage[lane];
        new_vertex<PREC>(S, nvt, kp, nr2, nX, nY, nZ, nf);
        mr = nr2;
    }
    // compact the kept triangles in place (destinations never pass sources)
    int dst = 0;
#pragma unroll 1
    for (int c = 0; c < nchunk; ++c) {
        const int t = c * 32 + lane;
        const bool keep = t < C.nt && !((outm.get(c) >> lane) & 1u);
        const unsigned km = __ballot_sync(FULL, keep);
        unsigned v = 0;
        long long r2 = 0;
        double x = 0, y = 0, z = 0;
        float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (keep) {
            v = S.tv[t];
            r2 = S.tr2[t];
            if constexpr (PREC == 0) { x = S.tx[t]; y = S.ty[t]; z = S.tz[t]; }
            else fv = S.tf[t];
        }
        __syncwarp();
        if (keep) {
            const int d = dst + __popc(km & lanemask_lt());
            mr = max(mr, r2);
            S.tv[d] = v;
            S.tr2[d] = r2;
            if constexpr (PREC == 0) { S.tx[d] = x; S.ty[d] = y; S.tz[d] = z; }
            else S.tf[d] = fv;
        }
        dst += __popc(km);
        __syncwarp();
    }
    // append the new vertices
    if (mk) {
        const int t = nkept + lane;
        S.tv[t] = nvt;
        S.tr2[t] = nr2;
        if constexpr (PREC == 0) { S.tx[t] = nX; S.ty[t] = nY; S.tz[t] = nZ; }
        else S.tf[t] = nf;
    }
    if constexpr (CAP::NS > 32) {
        // the large instance: new vertices beyond the first 32, one more per lane
        if (lane + 32 < nnew) {
            const unsigned v2 = S.stage[lane + 32];
            new_vertex<PREC>(S, v2, kp, nr2, nX, nY, nZ, nf);
            mr = max(mr, nr2);
            const int t = nkept + lane + 32;
            S.tv[t] = v2;
            S.tr2[t] = nr2;
            if constexpr (PREC == 0) { S.tx[t] = nX; S.ty[t] = nY; S.tz[t] = nZ; }
            else S.tf[t] = nf;
        }
    }
    __syncwarp();
    if (PREC == 0) C.solve64 += nnew;
    C.nt = nkept + nnew;
    C.np = max(C.np, kp + 1);
    C.cuts++;
    update_limit<PREC>(C, mr);
}

// What a flush needs besides the warp's shared memory to form the exact
// candidate planes: the binned generators (the image offsets s L - p of this
// generator are in shared memory).
struct Gather {
    const double4_32a *sorted;
};

// SORT 0 orders more than 32 candidates by a bitonic network on the buffer in
// shared memory, SORT 1 by the same network on keys held two per lane
// (shuffles, no barriers), producing only the permutation.  Both give the same
// order (the keys are unique), so the mesh does not depend on SORT; which is
// faster depends on the code around it, and the autotuner picks.
template <int PREC, class CAP, int SORT>
__device__ void flush_batch(ClipSmem<PREC, CAP> &S, int &ncand, CellState &C, int lane, const Gather &G)
{
    if (ncand == 0) return;
    // exact planes, one lane per candidate: q = r_j + s L - p in FP64 and the
    // bit pattern of |q|^2 (the sort key); the buffer held the sorted index.
    // A candidate at distance 0 is another generator at the same position: the
    // two cells coincide, which a Voronoi tessellation does not allow.
    bool coincident = false;
    for (int k = lane; k < ncand; k += 32) {
        const int code = S.csh[k];
        const double4_32a P = G.sorted[S.cid[k]];
        const int dx = code % 3, dy = (code / 3) % 3, dz = code / 9;
        const double qx = P.x + S.off[dx], qy = P.y + S.off[3 + dy], qz = P.z + S.off[6 + dz];
        S.u.c.x[k] = qx; S.u.c.y[k] = qy; S.u.c.z[k] = qz;
        const long long d2 = __double_as_longlong(__fma_rn(qx, qx, __fma_rn(qy, qy, __dmul_rn(qz, qz))));
        S.u.c.d2[k] = d2;
        coincident |= d2 == 0;
        S.cid[k] = (int)__double_as_longlong(P.w);
    }
    if (__any_sync(FULL, coincident)) {
        C.err |= ST_EDEGEN;
        ncand = 0;
        return;
    }
    __syncwarp();
    if (ncand <= 32) {
        // one candidate per lane: bitonic network on (|q|^2 bits, id, image)
        // with shuffles; the buffer stays in place and perm gives the order
        const bool have = lane < ncand;
        unsigned long long key = have ? (unsigned long long)S.u.c.d2[lane] : ~0ull;
        unsigned tie = have ? (unsigned)S.cid[lane] * 27u + (unsigned)S.csh[lane] : ~0u;
        int idx = lane;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int j = kk >> 1; j > 0; j >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(FULL, key, j);
                const unsigned ot = __shfl_xor_sync(FULL, tie, j);
                const int oi = __shfl_xor_sync(FULL, idx, j);
                const bool other_less = ok < key || (ok == key && ot < tie);
                const bool lower = (lane & j) == 0, up = (lane & kk) == 0;
                if (lower == up ? other_less : !other_less) { key = ok; tie = ot; idx = oi; }
            }
        }
        if (have) S.perm[lane] = (unsigned char)idx;
    } else if constexpr (SORT == 1) {
        // 33..64 candidates, two per lane (entries lane and lane + 32):
        // partners in other lanes by shuffles (distance below 32), in the
        // same lane at distance 32
        unsigned long long key0 = (unsigned long long)S.u.c.d2[lane];
        unsigned tie0 = (unsigned)S.cid[lane] * 27u + (unsigned)S.csh[lane];
        const bool have1 = lane + 32 < ncand;
        unsigned long long key1 = have1 ? (unsigned long long)S.u.c.d2[lane + 32] : ~0ull;
        unsigned tie1 = have1 ? (unsigned)S.cid[lane + 32] * 27u + (unsigned)S.csh[lane + 32] : ~0u;
        int idx0 = lane, idx1 = lane + 32;
#pragma unroll 1
        for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll 1
            for (int j = kk >> 1; j > 0; j >>= 1) {
                if (j == 32) {
                    // entries lane and lane + 32, ascending (kk = 64 here)
                    if (key1 < key0 || (key1 == key0 && tie1 < tie0)) {
                        const unsigned long long tk = key0; key0 = key1; key1 = tk;
                        const unsigned tt = tie0; tie0 = tie1; tie1 = tt;
                        const int ti = idx0; idx0 = idx1; idx1 = ti;
                    }
                    continue;
                }
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    unsigned long long &key = h ? key1 : key0;
                    unsigned &tie = h ? tie1 : tie0;
                    int &idx = h ? idx1 : idx0;
                    const unsigned long long ok = __shfl_xor_sync(FULL, key, j);
                    const unsigned ot = __shfl_xor_sync(FULL, tie, j);
                    const int oi = __shfl_xor_sync(FULL, idx, j);
                    const bool other_less = ok < key || (ok == key && ot < tie);
                    const bool up = ((lane + 32 * h) & kk) == 0;
                    if (lower == up ? other_less : !other_less) { key = ok; tie = ot; idx = oi; }
                }
            }
        }
        S.perm[lane] = (unsigned char)idx0;
        if (have1) S.perm[lane + 32] = (unsigned char)idx1;
    } else {
        sort_candidates(S, ncand, lane);
        for (int k = lane; k < ncand; k += 32) S.perm[k] = (unsigned char)k;
    }
    __syncwarp();
    if constexpr (PREC == 1) {
        // FP32 copies of the sorted planes, one lane per candidate
        for (int k = lane; k < ncand; k += 32) {
            S.u.c.cf[k] = make_float4((float)S.u.c.x[k], (float)S.u.c.y[k], (float)S.u.c.z[k],
                                      (float)half_of(S.u.c.d2[k]));
        }
        __syncwarp();
    }
    for (int k = 0; k < ncand; ++k) {
        const int kk = S.perm[k];
        if (S.u.c.d2[kk] > C.lim) break;
        clip_by<PREC, CAP>(S, kk, C, lane);
        if (C.err) break;
    }
    ncand = 0;
    __syncwarp();
}

// The main instance (CAP::BIG false) clips binned entry w of every warp; a
// cell that overflows one of its lists goes to the retry list instead of
// failing.  The large instance (one warp per block) clips entry retry[r] of
// block r and writes its faces to overflow row r.
template <int PREC, class CAP, int SORT>
__global__ void __maxnreg__(MM_CLIP_MAXNREG)
k_clip(const double4_32a *__restrict__ sorted, const float4 *__restrict__ sortedf, const int *__restrict__ start,
       int64_t n,
       const BoxDev *__restrict__ boxes, const int *__restrict__ cbox, double *__restrict__ vol,
       double *__restrict__ cen, Slots sl, DevStatus *st, int collect, int cand_cap)
{
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t w;
    bool strict = false;
    if constexpr (CAP::BIG) {
        const int nr = *(volatile int *)&st->nretry;
        if (blockIdx.x == 0 && threadIdx.x == 0 && nr > sl.orows) atomicOr(&st->flags, ST_ECAP_RETRY);
        if ((int64_t)blockIdx.x >= (nr < sl.orows ? (int64_t)nr : sl.orows)) return;
        const int e = sl.retry[blockIdx.x];
        strict = e < 0;
        w = strict ? ~e : e;
    } else {
        w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
        if (w >= n) return;
    }
    ClipSmem<PREC, CAP> &S = reinterpret_cast<ClipSmem<PREC, CAP> *>(dyn_smem)[wid];
    // A box's cells occupy the same range of indices in the input order and in
    // the binned order (the bins are laid out box by box), so the box of
    // binned entry w is cbox[w]: no need to wait for the generator's id.
    const BoxDev *const gp = boxes + cbox[w];  // for the lane-indexed fields
    const BoxDev g = *gp;
    const int self = (int)__double_as_longlong(sorted[w].w);
    const double amin = g.amin;
    // The setup runs in FP32 and integer arithmetic wherever a bound, not an
    // exact value, is needed: on GB300 an FP64 instruction costs the issue
    // time of dozens of FP32 ones.

    // starting box: planes 0..5 = +x,-x,+y,-y,+z,-z self-image bisectors
    if (lane < 6) {
        const int d = lane >> 1;
        const double L = gp->L[d];
        const double sL = (lane & 1) ? -L : L;
        S.px[lane] = d == 0 ? sL : 0.0;
        S.py[lane] = d == 1 ? sL : 0.0;
        S.pz[lane] = d == 2 ? sL : 0.0;
        S.po[lane] = half_of(__double_as_longlong(L * L));  // L^2 / 2
        S.pnb[lane] = self;
        int s3[3] = {0, 0, 0};
        s3[d] = (lane & 1) ? -1 : 1;
        S.psh[lane] = (s3[0] + 1) + 3 * (s3[1] + 1) + 9 * (s3[2] + 1);
        if constexpr (PREC == 1) {
            const float fo = (float)S.po[lane];
            const float Lf = gp->Lf[d];
            const float sLf = (lane & 1) ? -Lf : Lf;  // (float)(+-L)
            S.pf[lane] = make_float4(d == 0 ? sLf : 0.0f, d == 1 ? sLf : 0.0f, d == 2 ? sLf : 0.0f, fo);
            S.pfn[lane] = sqrtf(2.0f * fo);
        }
    } else if (lane < 15) {
        // image offsets s L - p of the three axes (lanes 6..14: axis, s)
        const int d = (lane - 6) / 3, s = (lane - 6) % 3;
        const double p = d == 0 ? sorted[w].x : (d == 1 ? sorted[w].y : sorted[w].z);
        const double L = gp->L[d];
        const double o = s == 1 ? -p : (s == 0 ? -L - p : L - p);
        S.off[lane - 6] = o;
        S.offf[lane - 6] = (float)o;
    }
    if (lane < 8) {
        // corner (sx, sy, sz): planes chosen by sign, ordered so det > 0
        const int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;  // 1 means negative
        unsigned a = sx, b = 2 + sy, c = 4 + sz;
        // det(sign_x e_x, sign_y e_y, sign_z e_z) = product of signs
        if ((sx ^ sy ^ sz) & 1) { unsigned t = b; b = c; c = t; }
        S.tv[lane] = a | (b << 8) | (c << 16);
        if constexpr (PREC == 0) {
            const double x = sx ? -0.5 * g.L[0] : 0.5 * g.L[0], y = sy ? -0.5 * g.L[1] : 0.5 * g.L[1],
                         z = sz ? -0.5 * g.L[2] : 0.5 * g.L[2];
            S.tr2[lane] = r2_bits64(x, y, z);
            S.tx[lane] = x; S.ty[lane] = y; S.tz[lane] = z;
        } else {
            // (float)(+-L/2) = +-Lf/2 exactly; |v|^2 from them in FP32, widened
            // past its rounding (an upper bound is all the limit needs)
            const float x = 0.5f * (sx ? -g.Lf[0] : g.Lf[0]), y = 0.5f * (sy ? -g.Lf[1] : g.Lf[1]),
                        z = 0.5f * (sz ? -g.Lf[2] : g.Lf[2]);
            S.tr2[lane] = (long long)__float_as_int(fmaf(x, x, fmaf(y, y, z * z)) * 1.000001f);
            S.tf[lane] = make_float4(x, y, z, 0.0f);
        }
    }
    for (int r = lane; r < CAP::BMW * CAP::PM; r += 32) S.bm[r] = 0u;
    __syncwarp();
    CellState C;
    C.np = 6;
    C.nt = 8;
    // 4 r_max^2 of the starting box is |L|^2: an FP32 upper bound of it
    C.lim = dbits_of_float(fmaf(g.Lf[0], g.Lf[0], fmaf(g.Lf[1], g.Lf[1], g.Lf[2] * g.Lf[2])) * 1.000001f);
    C.limk = __int_as_float(0x7f800000);  // keep everything until the first cut
    C.slack = 2e-6f * fmaxf(g.Lf[0], fmaxf(g.Lf[1], g.Lf[2]));
    C.err = 0;
    C.cuts = 0;
    C.strict = strict;
    C.pred64 = C.solve64 = C.fan64 = C.tested = 0;

    // Home bin of p in FP32 (the FP32 copy of p from the bin sort), and the
    // distance from p to the nearer wall of that bin per axis, lowered by the
    // slack (which exceeds the FP32 rounding of the whole computation): the
    // bins of rings 0..r then cover at least the radius min_d (edge_d + r bs_d),
    // also where rounding puts p just outside the bin.
    int cb[3];
    float edge[3];
    {
        const float4 mf = sortedf[w];
        const float pp[3] = {mf.x, mf.y, mf.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int c = (int)floorf(pp[d] * g.ibsf[d]);
            cb[d] = c < 0 ? 0 : (c >= g.g[d] ? g.g[d] - 1 : c);
            edge[d] = fminf(pp[d] - (float)cb[d] * g.bsf[d], (float)(cb[d] + 1) * g.bsf[d] - pp[d]) - C.slack;
        }
    }
    const Gather G{sorted};
    // The candidate gather is resumable: each lane walks the bins of the
    // current ring 32 at a time, the buffer is flushed (sorted and clipped)
    // whenever it cannot take another 32 candidates and at the end of every
    // ring, from one call site (one copy of the clipping code in the kernel).
    int ncand = 0, maxcand = 0;
    int rl = 0, rh = 1, total = 27, base = 0;
    int rings = 0;
    int cur = 0, end = 0, code = 13;
    float offx = 0.0f, offy = 0.0f, offz = 0.0f;
    bool selfimg = true;
    while (!C.err) {
        bool ring_done = false;
        while (ncand + 32 <= cand_cap) {
            if (!__any_sync(FULL, cur < end)) {
                if (base >= total) { ring_done = true; break; }
                // the next 32 bins of the ring, one per lane
                const int nb = 2 * rh + 1;
                const int t = base + lane;
                base += 32;
                cur = 0;
                end = 0;
                int shx = 0, shy = 0, shz = 0;
                if (t < total) {
                    int ox, oy, oz;
                    if (rh == 1) { ox = t % 3 - 1; oy = (t / 3) % 3 - 1; oz = t / 9 - 1; }
                    else if (rh == 2) { ox = t % 5 - 2; oy = (t / 5) % 5 - 2; oz = t / 25 - 2; }
                    else { const int3 o = ring_offset(t, nb, rh); ox = o.x; oy = o.y; oz = o.z; }
                    const int ch = max(abs(ox), max(abs(oy), abs(oz)));
                    if (ch >= rl) {
                        int bx = cb[0] + ox, by = cb[1] + oy, bz = cb[2] + oz;
                        // the image of a bin index: comparisons for the usual
                        // range [-g, 2g), a division beyond it (rings wider than the grid)
                        shx = (bx >= -g.g[0] && bx < 2 * g.g[0]) ? (bx < 0 ? -1 : (bx >= g.g[0] ? 1 : 0)) : floordiv(bx, g.g[0]);
                        shy = (by >= -g.g[1] && by < 2 * g.g[1]) ? (by < 0 ? -1 : (by >= g.g[1] ? 1 : 0)) : floordiv(by, g.g[1]);
                        shz = (bz >= -g.g[2] && bz < 2 * g.g[2]) ? (bz < 0 ? -1 : (bz >= g.g[2] ? 1 : 0)) : floordiv(bz, g.g[2]);
                        bx -= shx * g.g[0];
                        by -= shy * g.g[1];
                        bz -= shz * g.g[2];
                        const int b = g.bin_off + bx + g.g[0] * (by + g.g[1] * bz);
                        cur = start[b];
                        end = start[b + 1];
                        // images two or more boxes away never cut (positions lie in [0, L))
                        if (abs(shx) > 1 || abs(shy) > 1 || abs(shz) > 1) end = cur;
                    }
                }
                // FP32 offsets for the gather filter (the exact ones are formed at flush time)
                // (images two or more boxes away gather nothing: any offset will do)
                offx = S.offf[shx < 0 ? 0 : (shx > 0 ? 2 : 1)];
                offy = S.offf[3 + (shy < 0 ? 0 : (shy > 0 ? 2 : 1))];
                offz = S.offf[6 + (shz < 0 ? 0 : (shz > 0 ? 2 : 1))];
                code = (shx + 1) + 3 * (shy + 1) + 9 * (shz + 1);
                selfimg = (abs(shx) + abs(shy) + abs(shz)) <= 1;
                continue;
            }
            bool keep = false;
            const int idx = cur;
            if (cur < end) {
                const float4 Pf = sortedf[cur];
                ++cur;
                const float qx = Pf.x + offx, qy = Pf.y + offy, qz = Pf.z + offz;
                const float d2f = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
                // the generator itself is sorted entry w
                keep = !((int64_t)idx == w && selfimg) && d2f <= C.limk;
            }
            const unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                const int s = ncand + __popc(km & lanemask_lt());
                S.cid[s] = idx; S.csh[s] = code;
            }
            ncand += __popc(km);
            maxcand = max(maxcand, ncand);
            __syncwarp();
        }
        flush_batch<PREC, CAP, SORT>(S, ncand, C, lane, G);
        if (C.err || !ring_done) continue;
        ++rings;
        // radius the gathered rings are guaranteed to cover
        const float rr = (float)rh;
        const float R = fmaxf(fminf(fminf(fmaf(rr, g.bsf[0], edge[0]), fmaf(rr, g.bsf[1], edge[1])),
                                    fmaf(rr, g.bsf[2], edge[2])), 0.0f);
        if (C.lim <= dbits_of_float(R * R * 0.999999f)) break;  // R^2 rounded down
        rl = rh + 1;
        rh = rl;
        if (rh > CAP::MR) { C.err |= ST_ECAP_RING; break; }
        total = (2 * rh + 1) * (2 * rh + 1) * (2 * rh + 1);
        base = 0;
    }

    // ---- finalisation: FP64 vertices, faces, volume, centroid
    if (PREC == 1 && !C.err) {  // final FP64 vertices from their planes
        C.solve64 += C.nt;
        for (int t = lane; t < C.nt; t += 32) {
            const unsigned v = S.tv[t];
            double x, y, z;
            vertex64(S, v & 255u, (v >> 8) & 255u, (v >> 16) & 255u, x, y, z);
            S.tx[t] = x; S.ty[t] = y; S.tz[t] = z;
        }
        __syncwarp();
    }
    double vl = 0.0, vcx = 0.0, vcy = 0.0, vcz = 0.0;
    unsigned fan = 0;  // polygon edges summed (work counter)
    // Edge table for the face walk: every directed edge x -> y of a vertex
    // triangle (x, y, z) maps to that triangle and z, so the next vertex
    // around a face is one lookup.  Keys are unique in a closed
    // triangulation; the load stays below 3/4 (else the walk scans instead).
    // The first triangle of each face is the lowest index containing it.
    constexpr int ETAB = CAP::ETAB, PB = CAP::PB, TB = CAP::TB;
    const bool use_tab = !C.err && 3 * C.nt <= (3 * ETAB) / 4;
    unsigned *etab = S.u.f.etab;
    int *first = S.cid;  // the candidate ids are dead after clipping
    if (use_tab) {
        for (int i = lane; i < ETAB; i += 32) etab[i] = 0xffffffffu;
        for (int i = lane; i < C.np; i += 32) first[i] = 0x7fffffff;
        __syncwarp();
        for (int e = lane; e < 3 * C.nt; e += 32) {
            const int t = e / 3, k = e - 3 * (e / 3);
            const unsigned v = S.tv[t];
            const unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
            const unsigned x = k == 0 ? a : (k == 1 ? b : c);
            const unsigned y = k == 0 ? b : (k == 1 ? c : a);
            const unsigned z = k == 0 ? c : (k == 1 ? a : b);
            const unsigned key = (x << PB) | y;
            const unsigned ent = (key << (PB + TB)) | (z << TB) | (unsigned)t;
            unsigned h = (key * 2654435761u) >> CAP::EH;
            for (int probe = 0; probe < ETAB; ++probe) {
                if (atomicCAS(&etab[h], 0xffffffffu, ent) == 0xffffffffu) break;
                h = (h + 1) & (ETAB - 1);
            }
            atomicMin(&first[x], t);
        }
        __syncwarp();
    }
    if (!C.err) {
        for (int p = lane; p < C.np; p += 32) {
            int t0 = -1;
            unsigned y = 0;
            if (use_tab) {
                const int f0 = first[p];
                if (f0 != 0x7fffffff) {
                    t0 = f0;
                    const unsigned v = S.tv[t0];
                    const unsigned a = v & 255u, b = (v >> 8) & 255u, c = (v >> 16) & 255u;
                    y = a == (unsigned)p ? c : (b == (unsigned)p ? a : b);
                }
            } else {
                t0 = scan_first(S.tv, C.nt, (unsigned)p, y);
            }
            S.u.f.a[p] = 0.0;
            if (t0 < 0) continue;  // plane no longer bounds the cell
            // Fan about the polygon's first vertex v0 with offsets d = v - v0
            // formed once per vertex.  The offsets lie in the plane x.q = o,
            // so d_a x d_b is parallel to q and q . (d_a x d_b) equals
            // (|q|^2 / q_k) times the 2-D cross product of the two coordinates
            // other than k, the axis where |q| is largest.  Edge (a, b) spans
            // the triangle (v0, a, b) with 2-D weight w; with W = sum w:
            // area = |W| |q| / (2 |q_k|), pyramid volume A |q| / 6 =
            // |W| |q|^2 / (12 |q_k|), centroid offset = sum w (d_a + d_b) / (3 W)
            // in the two kept coordinates, and in the k-th from the plane
            // equation q . offset = 0.  Offsets from v0 keep the rounding
            // relative to the face's own size.
            const double qx = S.px[p], qy = S.py[p], qz = S.pz[p];
            const long long aqx = abs_bits(qx), aqy = abs_bits(qy), aqz = abs_bits(qz);
            const int k = (aqx >= aqy && aqx >= aqz) ? 0 : (aqy >= aqz ? 1 : 2);
            const double *T1 = k == 0 ? S.ty : S.tx;  // kept coordinates (u, v)
            const double *T2 = k == 2 ? S.ty : S.tz;
            const double qk = k == 0 ? qx : (k == 1 ? qy : qz);
            const double q1 = k == 0 ? qy : qx, q2 = k == 2 ? qy : qz;
            const double u0 = T1[t0], v0 = T2[t0];
            double au = 0.0, av = 0.0;  // offset of the current vertex
            double W = 0.0, su = 0.0, sv = 0.0;
            int cnt = 0;
            bool ok = false;
            for (int guard = 0; guard < CAP::TM; ++guard) {
                // next vertex around p: the triangle containing p -> y
                int tn = -1;
                unsigned z = 0;
                if (use_tab) {
                    const unsigned key = ((unsigned)p << PB) | y;
                    unsigned h = (key * 2654435761u) >> CAP::EH;
                    for (int probe = 0; probe < ETAB; ++probe) {
                        const unsigned ent = etab[h];
                        if (ent == 0xffffffffu) break;
                        if ((ent >> (PB + TB)) == key) {
                            tn = (int)(ent & ((1u << TB) - 1u));
                            z = (ent >> TB) & ((1u << PB) - 1u);
                            break;
                        }
                        h = (h + 1) & (ETAB - 1);
                    }
                } else {
                    tn = scan_next(S.tv, C.nt, (unsigned)p, y, z);
                }
                if (tn < 0) break;
                ++cnt;
                if (tn == t0) { ok = true; break; }
                const double bu = T1[tn] - u0, bv = T2[tn] - v0;
                const double w = au * bv - av * bu;
                W += w;
                su += w * (au + bu);
                sv += w * (av + bv);
                au = bu; av = bv;
                y = z;
            }
            fan += cnt;
            if (!ok) { C.err |= ST_EDEGEN_CUT; continue; }
            const double aw = fabs(W);
            const double qn2 = 2.0 * S.po[p];  // |q|^2
            // 1 / q_k and 1 / (3 W) from one reciprocal of 3 W q_k; a face
            // of zero fan weight (area 0) takes 0 for both
            const double w3 = 3.0 * W;
            const bool nz = abs_bits(W) != 0;
            const double r = nz ? 1.0 / (w3 * qk) : 0.0;
            const double iq = w3 * r, iqk = fabs(iq);
            const double area = 0.5 * aw * (qn2 * rsqrt(qn2)) * iqk;
            const double i3w = qk * r;
            const double du = su * i3w, dv = sv * i3w;
            const double dk = -(q1 * du + q2 * dv) * iq;
            const double fx = S.tx[t0] + (k == 0 ? dk : du);
            const double fy = S.ty[t0] + (k == 1 ? dk : (k == 0 ? du : dv));
            const double fz = S.tz[t0] + (k == 2 ? dk : dv);
            S.u.f.a[p] = area;
            S.u.f.x[p] = fx; S.u.f.y[p] = fy; S.u.f.z[p] = fz;
            const double vp = aw * qn2 * iqk * (1.0 / 12.0);
            vl += vp;
            vcx += 0.75 * vp * fx;
            vcy += 0.75 * vp * fy;
            vcz += 0.75 * vp * fz;
        }
        C.err = __reduce_or_sync(FULL, (unsigned)C.err);
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fan += __shfl_xor_sync(FULL, fan, o);
    warp_sum4(vl, vcx, vcy, vcz, lane);

    int nface = 0;
    if (!C.err) {
        // the main instance writes row `self` of the per-cell slots, the large
        // one overflow row blockIdx.x
        int *const rnb = CAP::BIG ? sl.onb : sl.nb;
        unsigned char *const rsh = CAP::BIG ? sl.osh : sl.sh;
        double *const rarea = CAP::BIG ? sl.oarea : sl.area;
        double *const rfc = CAP::BIG ? sl.ofc : sl.fc;
        const int64_t sbase = CAP::BIG ? (int64_t)blockIdx.x * CAP::MF : (int64_t)self * CAP::MF;
        const int64_t ns = CAP::BIG ? sl.orows * (int64_t)CAP::MF : n * (int64_t)CAP::MF;
        for (int p0 = 0; p0 < C.np; p0 += 32) {
            const int p = p0 + lane;
            const bool keep = p < C.np && abs_bits(S.u.f.a[p]) > abs_bits(amin);  // both >= 0
            const unsigned km = __ballot_sync(FULL, keep);
            if (keep) {
                const int k = nface + __popc(km & lanemask_lt());
                if (k < CAP::MF) {
                    const int64_t s = sbase + k;
                    rnb[s] = S.pnb[p];
                    rsh[s] = (unsigned char)S.psh[p];
                    rarea[s] = S.u.f.a[p];
                    rfc[s] = S.u.f.x[p];  // relative to the generator
                    rfc[ns + s] = S.u.f.y[p];
                    rfc[2 * ns + s] = S.u.f.z[p];
                }
            }
            nface += __popc(km);
        }
        if (nface > CAP::MF) C.err |= ST_ECAP_FACE;
    }
    if (lane == 0) {
        if (C.err) {
            nface = 0;
            if (!CAP::BIG && (C.err & ~ST_RETRYABLE) == 0) {
                // over a capacity of this instance, or an inconsistent cut: the
                // large one clips it again (with the strict tie rule for the latter)
                sl.retry[atomicAdd(&st->nretry, 1)] = (C.err & ST_EDEGEN_CUT) ? ~(int)w : (int)w;
            } else {
                atomicOr(&st->flags, C.err);
                atomicExch(&st->bad_cell, self);
            }
        }
        if constexpr (CAP::BIG) {
            sl.ocnt[blockIdx.x] = nface;
            sl.cnt[self] = C.err ? 0 : -(int)blockIdx.x - 1;
        } else {
            sl.cnt[self] = nface;
        }
        // volume and first moment about the generator; the face kernel turns
        // the moment into the centroid (one thread per cell, off this warp)
        vol[self] = vl;
        cen[self] = vcx;
        cen[n + self] = vcy;
        cen[2 * n + self] = vcz;
        if (collect) {
            atomicMax(&st->max_cand, maxcand);
            atomicMax(&st->max_planes, C.np);
            atomicMax(&st->max_tris, C.nt);
            if (rings > 1) atomicAdd(&st->multi_ring, 1);
            atomicAdd(&st->cuts, (unsigned long long)C.cuts);
            atomicAdd(&st->pred64, (unsigned long long)C.pred64);
            atomicAdd(&st->solve64, (unsigned long long)C.solve64);
            atomicAdd(&st->fan64, (unsigned long long)fan);
            atomicAdd(&st->tested, (unsigned long long)C.tested);
        }
    }
}

template <int PREC, class CAP, int SORT>
static void launch_clip_t(const double4_32a *sorted, const float4 *sortedf, const int *start, int64_t n,
                          const BoxDev *boxes, const int *cbox, double *vol, double *cen, Slots sl, DevStatus *st,
                          int collect, int warps, int cand_cap, int64_t blocks, cudaStream_t s)
{
    static bool configured = false;  // the attribute is per function and process-wide
    if (!configured) {
        cudaFuncSetAttribute(k_clip<PREC, CAP, SORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(ClipSmem<PREC, CAP>) * (CAP::BIG ? 1 : CLIP_MAX_WARPS)));
        configured = true;
    }
    const size_t smem = sizeof(ClipSmem<PREC, CAP>) * warps;
    k_clip<PREC, CAP, SORT><<<(unsigned)blocks, 32 * warps, smem, s>>>(sorted, sortedf, start, n, boxes, cbox, vol, cen,
                                                                 sl, st, collect, cand_cap);
}

void launch_clip(const double4_32a *sorted, const float4 *sortedf, const int *start, int64_t n, const BoxDev *boxes,
                 const int *cbox,
                 int precision, int collect, int warps, int cand_cap, int sort, double *vol, double *cen,
                 Slots sl, DevStatus *st, cudaStream_t s)
{
    warps = warps < 1 ? 1 : (warps > CLIP_MAX_WARPS ? CLIP_MAX_WARPS : warps);
    cand_cap = cand_cap < 32 ? 32 : (cand_cap > CBATCH ? CBATCH : cand_cap);
    const int64_t nb = (n + warps - 1) / warps;
    // the sort variant only changes speed, so the direct FP64 clipper keeps one
    if (precision == 0)
        launch_clip_t<0, CapMain, 0>(sorted, sortedf, start, n, boxes, cbox, vol, cen, sl, st, collect, warps, cand_cap, nb, s);
    else if (sort == 1)
        launch_clip_t<1, CapMain, 1>(sorted, sortedf, start, n, boxes, cbox, vol, cen, sl, st, collect, warps, cand_cap, nb, s);
    else
        launch_clip_t<1, CapMain, 0>(sorted, sortedf, start, n, boxes, cbox, vol, cen, sl, st, collect, warps, cand_cap, nb, s);
}

void launch_clip_big(const double4_32a *sorted, const float4 *sortedf, const int *start, int64_t n,
                     const BoxDev *boxes, const int *cbox, int precision, int collect, int cand_cap, double *vol,
                     double *cen, Slots sl, DevStatus *st, cudaStream_t s)
{
    if (sl.orows < 1) return;
    cand_cap = cand_cap < 32 ? 32 : (cand_cap > CBATCH ? CBATCH : cand_cap);
    if (precision == 0)
        launch_clip_t<0, CapBig, 0>(sorted, sortedf, start, n, boxes, cbox, vol, cen, sl, st, collect, 1, cand_cap, sl.orows, s);
    else
        launch_clip_t<1, CapBig, 0>(sorted, sortedf, start, n, boxes, cbox, vol, cen, sl, st, collect, 1, cand_cap, sl.orows, s);
}

}  // namespace mm
