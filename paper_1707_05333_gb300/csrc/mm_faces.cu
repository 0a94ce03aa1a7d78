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

static_assert(MAXF % 4 == 0, "slot rows are read as int4");

// Per cell: find the partner slot of each face in the neighbour's list,
// then mark which faces are confirmed and which this cell stores.
__global__ void k_face_confirm(int64_t n, Slots sl, unsigned long long *__restrict__ emit_mask,
                               unsigned long long *__restrict__ conf_mask, signed char *__restrict__ partner,
                               int *__restrict__ emit_cnt, int *__restrict__ conf_cnt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cnt = sl.cnt[i];
    unsigned long long em = 0, cm = 0;
    for (int k = 0; k < cnt; ++k) {
        const int64_t s = i * MAXF + k;
        const int j = sl.nb[s];
        const int code = sl.sh[s];
        const int want = 26 - code;  // the mirrored image seen from j
        const int cj = sl.cnt[j];
        int m = -1;
        // the neighbour's slots four at a time (rows of MAXF ints are 16-byte aligned)
        const int4 *row = reinterpret_cast<const int4 *>(sl.nb + (int64_t)j * MAXF);
        for (int t0 = 0; t0 < cj && m < 0; t0 += 4) {
            const int4 q = row[t0 >> 2];
            const int c4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int t = t0 + a;
                if (m < 0 && t < cj && c4[a] == (int)i && sl.sh[(int64_t)j * MAXF + t] == want) m = t;
            }
        }
        partner[s] = (signed char)m;
        if (m >= 0) {
            cm |= 1ull << k;
            if (i < j || (i == j && code > 13)) em |= 1ull << k;
        }
    }
    emit_mask[i] = em;
    conf_mask[i] = cm;
    emit_cnt[i] = __popcll(em);
    conf_cnt[i] = __popcll(cm);
}

// One warp per cell, one lane per face slot: the slot rows are read and the
// face records and incidences written with consecutive lanes on consecutive
// addresses.  Each slot knows its place in the face and incidence lists from
// the masks, so the results do not depend on the schedule.
__global__ void k_face_write(int64_t n, const double *__restrict__ pos, const BoxDev *__restrict__ boxes,
                             const int *__restrict__ cbox, Slots sl,
                             const unsigned long long *__restrict__ emit_mask,
                             const unsigned long long *__restrict__ conf_mask,
                             const signed char *__restrict__ partner, const int *__restrict__ face_off,
                             const int *__restrict__ inc_off, int *__restrict__ face_i, int *__restrict__ face_j,
                             int *__restrict__ face_shift, double *__restrict__ face_area,
                             double *__restrict__ face_normal, double *__restrict__ face_cen, int64_t fcap,
                             int *__restrict__ inc_face, int64_t icap, const double *__restrict__ vol,
                             double *__restrict__ cen, DevStatus *st)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;  // whole warps
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
    const unsigned long long em = emit_mask[i], cm = conf_mask[i];
    const int fbase = face_off[i], e0 = inc_off[i];
    const int64_t ns = n * (int64_t)MAXF;
    const int kend = 64 - __clzll((long long)cm);
    for (int k = lane; k < kend; k += 32) {
        if (!((cm >> k) & 1ull)) continue;
        const int e = e0 + __popcll(cm & ((1ull << k) - 1ull));
        const int64_t s = i * MAXF + k;
        const int j = sl.nb[s];
        const int code = sl.sh[s];
        if ((em >> k) & 1ull) {
            const int f = fbase + __popcll(em & ((1ull << k) - 1ull));
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
                face_area[f] = sl.area[s];
                face_normal[f] = qx * inv;
                face_normal[fcap + f] = qy * inv;
                face_normal[2 * fcap + f] = qz * inv;
                face_cen[f] = pix + sl.fc[s];  // the slots hold it relative to the generator
                face_cen[fcap + f] = piy + sl.fc[ns + s];
                face_cen[2 * fcap + f] = piz + sl.fc[2 * ns + s];
            }
            inc_face[e] = f;
        } else {
            const int m = partner[s];
            const unsigned long long ej = emit_mask[j];
            const int f = face_off[j] + __popcll(ej & ((1ull << m) - 1ull));
            inc_face[e] = ~f;
        }
    }
}

void launch_face_confirm(int64_t n, Slots sl, unsigned long long *emit_mask, unsigned long long *conf_mask,
                         signed char *partner, int *emit_cnt, int *conf_cnt, cudaStream_t s)
{
    int nb = (int)((n + 127) / 128);
    k_face_confirm<<<nb, 128, 0, s>>>(n, sl, emit_mask, conf_mask, partner, emit_cnt, conf_cnt);
}

void launch_face_write(int64_t n, const double *pos, const BoxDev *boxes, const int *cbox, Slots sl,
                       const unsigned long long *emit_mask, const unsigned long long *conf_mask,
                       const signed char *partner, const int *face_off, const int *inc_off, int *face_i,
                       int *face_j, int *face_shift, double *face_area, double *face_normal, double *face_cen,
                       int64_t fcap, int *inc_face, int64_t icap, const double *vol, double *cen, DevStatus *st,
                       cudaStream_t s)
{
    const int nb = (int)((n + 3) / 4);  // four cells (warps) per block
    k_face_write<<<nb, 128, 0, s>>>(n, pos, boxes, cbox, sl, emit_mask, conf_mask, partner, face_off, inc_off,
                                    face_i, face_j, face_shift, face_area, face_normal, face_cen, fcap, inc_face,
                                    icap, vol, cen, st);
}

}  // namespace mm
