// mm_faces.cu -- unique faces and the per-cell incident-face lists.
//
// Every shared face was written twice by the clipper, once from each side.
// A face counts only if both sides have it (so the two cells always agree on
// their neighbours); it is stored once, by the cell with the smaller index,
// or, for a cell touching its own periodic image, by the copy whose image
// code is above the zero-shift code.  Offsets come from exclusive scans of
// per-cell counts, so face ids and every cell's incident list are
// deterministic: no atomics on the data path.
#include "mm_internal.cuh"

namespace mm {

static_assert(MAXF % 4 == 0 && MAXF_BIG % 4 == 0, "slot rows are read as int4");
static_assert(MAXF <= 64 && MAXF_BIG <= 128, "face masks hold one word per 64 slots, at most two");
// Lanes sharing one cell's slots in the confirmation (the partner searches
// are independent).  Measured on the 256^3 shear layer, face stage per
// tessellation: one thread per cell 10.06 ms, 2 lanes 9.70, 4 lanes 9.82,
// 8 lanes 10.29.
constexpr int CONFIRM_LANES = 2;

// The face slots of one cell: its row of the main slot arrays, or, for a
// cell the large clipper re-clipped, its overflow row.
struct Row {
    const int *nb;
    const unsigned char *sh;
    const double *area, *fc;
    int64_t base, fstride;  // first slot; row stride of the [3][.] centroid array
    int cnt, orow;          // faces; overflow row or -1
};

__device__ __forceinline__ Row row_of(const Slots &sl, int64_t n, int64_t i)
{
    Row r;
    const int c = sl.cnt[i];
    if (c >= 0) {
        r.nb = sl.nb; r.sh = sl.sh; r.area = sl.area; r.fc = sl.fc;
        r.base = i * MAXF;
        r.fstride = n * (int64_t)MAXF;
        r.cnt = c;
        r.orow = -1;
    } else {
        const int k = -c - 1;
        r.nb = sl.onb; r.sh = sl.osh; r.area = sl.oarea; r.fc = sl.ofc;
        r.base = (int64_t)k * MAXF_BIG;
        r.fstride = sl.orows * (int64_t)MAXF_BIG;
        r.cnt = sl.ocnt[k];
        r.orow = k;
    }
    return r;
}

// Number of set bits of the two-word mask below bit k.
__device__ __forceinline__ int popc_below(unsigned long long m0, unsigned long long m1, int k)
{
    if (k < 64) return __popcll(m0 & ((1ull << k) - 1ull));
    return __popcll(m0) + __popcll(m1 & ((1ull << (k - 64)) - 1ull));
}

// The slot of row (nb, sh) holding neighbour i seen through image `want`, or
// -1; the row's ids are read four at a time (rows are 16-byte aligned).
__device__ __forceinline__ int find_partner(const int *nb, const unsigned char *sh, int cnt, int i, int want)
{
    int m = -1;
    const int4 *row = reinterpret_cast<const int4 *>(nb);
    for (int t0 = 0; t0 < cnt && m < 0; t0 += 4) {
        const int4 v = row[t0 >> 2];
        const int c4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int t = t0 + a;
            if (m < 0 && t < cnt && c4[a] == i && sh[t] == want) m = t;
        }
    }
    return m;
}

// Per cell: find the partner slot of each face in the neighbour's list,
// then mark which faces are confirmed and which this cell stores.  The
// CONFIRM_LANES lanes of a cell take every CONFIRM_LANES-th slot from `lane`
// and OR their bits together; lane 0 writes the masks.  A cell in
// an overflow row keeps two mask words there; the low word also goes to the
// per-cell mask, which is all a neighbour's partner slot below 64 needs.
// OVF false: no cell was re-clipped, every row is a main row.
//
// A face the neighbour does not confirm is dropped, which is right for the
// faces near the area threshold that one side keeps and the other drops.  A
// face far above it (1e4 times the threshold) that the neighbour lacks means
// the two cells disagree on the mesh (near-degenerate generators): that is
// reported (ST_EDEGEN_CUT, cell i) instead of returned.
template <bool OVF>
__device__ __forceinline__ void face_confirm_cell(int64_t n, int64_t i, int lane, const Slots &sl, const OvfFaces &ov,
                                                  double amin, DevStatus *st,
                                                  unsigned long long *__restrict__ emit_mask,
                                                  unsigned long long *__restrict__ conf_mask,
                                                  signed char *__restrict__ partner, int *__restrict__ emit_cnt,
                                                  int *__restrict__ conf_cnt)
{
    Row r;
    if constexpr (OVF) {
        r = row_of(sl, n, i);
    } else {
        r.nb = sl.nb; r.sh = sl.sh; r.area = sl.area; r.base = i * MAXF; r.cnt = sl.cnt[i]; r.orow = -1;
    }
    signed char *const part = (!OVF || r.orow < 0) ? partner : ov.partner;
    unsigned long long em0 = 0, cm0 = 0, em1 = 0, cm1 = 0;
    for (int k = lane; k < r.cnt; k += CONFIRM_LANES) {
        const int64_t s = r.base + k;
        const int j = r.nb[s];
        const int code = r.sh[s];
        const int want = 26 - code;  // the mirrored image seen from j
        const int cj = sl.cnt[j];
        int m;
        if (!OVF || cj >= 0) {
            m = find_partner(sl.nb + (int64_t)j * MAXF, sl.sh + (int64_t)j * MAXF, cj, (int)i, want);
        } else {
            const int64_t ob = (int64_t)(-cj - 1) * MAXF_BIG;
            m = find_partner(sl.onb + ob, sl.osh + ob, sl.ocnt[-cj - 1], (int)i, want);
        }
        part[s] = (signed char)m;
        if (m < 0 && amin > 0.0 && r.area[s] > 1e4 * amin) {
            atomicOr(&st->flags, ST_EDEGEN_CUT);
            atomicExch(&st->bad_cell, (int)i);
        }
        if (m >= 0) {
            const unsigned long long bit = 1ull << (k & 63);
            const bool mine = i < j || (i == j && code > 13);
            if (!OVF || k < 64) {
                cm0 |= bit;
                if (mine) em0 |= bit;
            } else {
                cm1 |= bit;
                if (mine) em1 |= bit;
            }
        }
    }
    // the lanes of the cell combine their faces' bits
#pragma unroll
    for (int o = 1; o < CONFIRM_LANES; o <<= 1) {
        em0 |= __shfl_xor_sync(0xffffffffu, em0, o);
        cm0 |= __shfl_xor_sync(0xffffffffu, cm0, o);
        if (OVF) {
            em1 |= __shfl_xor_sync(0xffffffffu, em1, o);
            cm1 |= __shfl_xor_sync(0xffffffffu, cm1, o);
        }
    }
    if (lane != 0) return;
    emit_mask[i] = em0;
    conf_mask[i] = cm0;
    if (OVF && r.orow >= 0) {
        ov.emit[2 * r.orow] = em0;
        ov.emit[2 * r.orow + 1] = em1;
        ov.conf[2 * r.orow] = cm0;
        ov.conf[2 * r.orow + 1] = cm1;
    }
    emit_cnt[i] = __popcll(em0) + (OVF ? __popcll(em1) : 0);
    conf_cnt[i] = __popcll(cm0) + (OVF ? __popcll(cm1) : 0);
}

__global__ void k_face_confirm(int64_t n, Slots sl, OvfFaces ov, const BoxDev *__restrict__ boxes,
                               const int *__restrict__ cbox, DevStatus *st, unsigned long long *__restrict__ emit_mask,
                               unsigned long long *__restrict__ conf_mask, signed char *__restrict__ partner,
                               int *__restrict__ emit_cnt, int *__restrict__ conf_cnt)
{
    // CONFIRM_LANES lanes per cell; a group past n takes no slot but joins the shuffles
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / CONFIRM_LANES;
    const int lane = threadIdx.x % CONFIRM_LANES;
    const int64_t i = g < n ? g : n - 1;
    const bool live = g < n;
    const double amin = boxes[cbox[i]].amin;
    if (*ov.nretry == 0) face_confirm_cell<false>(n, i, live ? lane : MAXF_BIG, sl, ov, amin, st, emit_mask,
                                                  conf_mask, partner, emit_cnt, conf_cnt);
    else face_confirm_cell<true>(n, i, live ? lane : MAXF_BIG, sl, ov, amin, st, emit_mask, conf_mask, partner,
                                 emit_cnt, conf_cnt);
}

// The face records and incidences of cell i's confirmed slots, one lane per
// slot (OVF false: no cell was re-clipped, every row is a main row).
template <bool OVF>
__device__ __forceinline__ void face_write_slots(int64_t n, int64_t i, int lane, int stride, double pix, double piy,
                                                 double piz,
                                                 const double *L, const double *__restrict__ pos, const Slots &sl,
                                                 const OvfFaces &ov, const unsigned long long *__restrict__ emit_mask,
                                                 const unsigned long long *__restrict__ conf_mask,
                                                 const signed char *__restrict__ partner,
                                                 const int *__restrict__ face_off, const int *__restrict__ inc_off,
                                                 int *__restrict__ face_i, int *__restrict__ face_j,
                                                 int *__restrict__ face_shift, double *__restrict__ face_area,
                                                 double *__restrict__ face_normal, double *__restrict__ face_cen,
                                                 int64_t fcap, int *__restrict__ inc_face)
{
    Row r;
    if constexpr (OVF) {
        r = row_of(sl, n, i);
    } else {
        r.nb = sl.nb; r.sh = sl.sh; r.area = sl.area; r.fc = sl.fc;
        r.base = i * MAXF; r.fstride = n * (int64_t)MAXF; r.orow = -1;
    }
    const unsigned long long em0 = emit_mask[i], cm0 = conf_mask[i];
    unsigned long long em1 = 0, cm1 = 0;
    if (OVF && r.orow >= 0) {
        em1 = ov.emit[2 * r.orow + 1];
        cm1 = ov.conf[2 * r.orow + 1];
    }
    const int fbase = face_off[i], e0 = inc_off[i];
    const int kend = cm1 ? 128 - __clzll((long long)cm1) : 64 - __clzll((long long)cm0);
    for (int k = lane; k < kend; k += stride) {
        if (!(((k < 64 ? cm0 : cm1) >> (k & 63)) & 1ull)) continue;
        const int e = e0 + (OVF ? popc_below(cm0, cm1, k) : __popcll(cm0 & ((1ull << k) - 1ull)));
        const int64_t s = r.base + k;
        const int j = r.nb[s];
        const int code = r.sh[s];
        if ((((k < 64 ? em0 : em1) >> (k & 63)) & 1ull)) {
            const int f = fbase + (OVF ? popc_below(em0, em1, k) : __popcll(em0 & ((1ull << k) - 1ull)));
            if (f < fcap) {
                // image offsets -L, 0, +L by selection (no FP64 arithmetic)
                const int cx = code % 3, cy = (code / 3) % 3, cz = code / 9;
                const double ox = cx == 1 ? 0.0 : (cx == 2 ? L[0] : -L[0]);
                const double oy = cy == 1 ? 0.0 : (cy == 2 ? L[1] : -L[1]);
                const double oz = cz == 1 ? 0.0 : (cz == 2 ? L[2] : -L[2]);
                const double qx = pos[j] + ox - pix;
                const double qy = pos[n + j] + oy - piy;
                const double qz = pos[2 * n + j] + oz - piz;
                const double inv = rsqrt(qx * qx + qy * qy + qz * qz);
                face_i[f] = (int)i;
                face_j[f] = j;
                face_shift[f] = code;
                face_area[f] = r.area[s];
                face_normal[f] = qx * inv;
                face_normal[fcap + f] = qy * inv;
                face_normal[2 * fcap + f] = qz * inv;
                face_cen[f] = pix + r.fc[s];  // the slots hold it relative to the generator
                face_cen[fcap + f] = piy + r.fc[r.fstride + s];
                face_cen[2 * fcap + f] = piz + r.fc[2 * r.fstride + s];
            }
            inc_face[e] = f;
        } else {
            const int m = ((!OVF || r.orow < 0) ? partner : ov.partner)[s];
            int pre;
            if (!OVF || m < 64) {
                pre = __popcll(emit_mask[j] & ((1ull << m) - 1ull));
            } else {  // a slot of the second word: j's faces are in an overflow row
                const int kj = -sl.cnt[j] - 1;
                pre = popc_below(ov.emit[2 * kj], ov.emit[2 * kj + 1], m);
            }
            inc_face[e] = ~(face_off[j] + pre);
        }
    }
}

// Four lanes per cell, each taking every fourth face slot: eight cells per
// warp keep the lanes busy (a cell has about 16 faces; a warp per cell left
// half the lanes idle and its FP64 work per face made that the bound;
// measured at 256^3: a warp 18.4 ms, 16 lanes 14.3, 8 lanes 11.4, 4 lanes
// 10.1, 2 lanes 9.9, one thread 21.0; on random points 4 lanes was best).
// Each slot knows its place in the face and incidence lists from the masks,
// so the results do not depend on the schedule.
__global__ void k_face_write(int64_t n, const double *__restrict__ pos, const BoxDev *__restrict__ boxes,
                             const int *__restrict__ cbox, Slots sl, OvfFaces ov,
                             const unsigned long long *__restrict__ emit_mask,
                             const unsigned long long *__restrict__ conf_mask,
                             const signed char *__restrict__ partner, const int *__restrict__ face_off,
                             const int *__restrict__ inc_off, int *__restrict__ face_i, int *__restrict__ face_j,
                             int *__restrict__ face_shift, double *__restrict__ face_area,
                             double *__restrict__ face_normal, double *__restrict__ face_cen, int64_t fcap,
                             int *__restrict__ inc_face, int64_t icap, const double *__restrict__ vol,
                             double *__restrict__ cen, DevStatus *st)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2;
    const int lane = threadIdx.x & 3;
    if (i >= n) return;  // whole groups of four lanes
    const double pix = pos[i], piy = pos[n + i], piz = pos[2 * n + i];
    if (lane == 0) {
        // the cell centroid from the clipper's volume and first moment about
        // the generator
        const double ivl = 1.0 / vol[i];
        cen[i] = pix + cen[i] * ivl;
        cen[n + i] = piy + cen[n + i] * ivl;
        cen[2 * n + i] = piz + cen[2 * n + i] * ivl;
    }
    const double *L = boxes[cbox[i]].L;
    // a fixed capacity (graph mode) that is too small is reported, never overrun
    if ((int64_t)face_off[i + 1] > fcap || (int64_t)inc_off[i + 1] > icap) {
        if (lane == 0) atomicOr(&st->flags, ST_ECAP_MESH);
        return;
    }
    if (*ov.nretry == 0)
        face_write_slots<false>(n, i, lane, 4, pix, piy, piz, L, pos, sl, ov, emit_mask, conf_mask, partner,
                                face_off, inc_off, face_i, face_j, face_shift, face_area, face_normal, face_cen, fcap,
                                inc_face);
    else
        face_write_slots<true>(n, i, lane, 4, pix, piy, piz, L, pos, sl, ov, emit_mask, conf_mask, partner,
                               face_off, inc_off, face_i, face_j, face_shift, face_area, face_normal, face_cen, fcap,
                               inc_face);
}

void launch_face_confirm(int64_t n, Slots sl, OvfFaces ov, const BoxDev *boxes, const int *cbox, DevStatus *st,
                         unsigned long long *emit_mask, unsigned long long *conf_mask, signed char *partner,
                         int *emit_cnt, int *conf_cnt, cudaStream_t s)
{
    const int64_t nb = (n * CONFIRM_LANES + 127) / 128;
    k_face_confirm<<<(unsigned)nb, 128, 0, s>>>(n, sl, ov, boxes, cbox, st, emit_mask, conf_mask, partner, emit_cnt,
                                                conf_cnt);
}

void launch_face_write(int64_t n, const double *pos, const BoxDev *boxes, const int *cbox, Slots sl, OvfFaces ov,
                       const unsigned long long *emit_mask, const unsigned long long *conf_mask,
                       const signed char *partner, const int *face_off, const int *inc_off, int *face_i,
                       int *face_j, int *face_shift, double *face_area, double *face_normal, double *face_cen,
                       int64_t fcap, int *inc_face, int64_t icap, const double *vol, double *cen, DevStatus *st,
                       cudaStream_t s)
{
    const int nb = (int)((n + 31) / 32);  // 32 cells per block of 128 threads
    k_face_write<<<nb, 128, 0, s>>>(n, pos, boxes, cbox, sl, ov, emit_mask, conf_mask, partner, face_off, inc_off,
                                    face_i, face_j, face_shift, face_area, face_normal, face_cen, fcap, inc_face,
                                    icap, vol, cen, st);
}

}  // namespace mm
