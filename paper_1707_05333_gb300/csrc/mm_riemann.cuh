// mm_riemann.cuh -- the face-frame Riemann solver and floors shared by the
// FP64 and the mixed-precision hydro kernels (Sec. 4, Sec. 4.1).
#pragma once

namespace mm {

// Wave speeds of a face's Riemann problem along the unit normal, for the
// entropy column's flux and shock Mach number (Sec. 4.3): Davis S_L, S_R, the
// contact speed S* and the normal velocities u_L, u_R.
template <class T>
struct WavesT {
    T sl, sr, ss, ul, ur;
};

template <class T>
struct FaceStateT {
    T rho, vx, vy, vz, P;  // velocity already in the face frame
    T irho;                // 1 / rho (formed once per face state)
};

// Order-preserving map of a double onto a signed 64-bit integer (the
// sign-magnitude bit pattern turned into two's complement), its own inverse:
// comparisons of doubles as integers take integer instructions instead of
// FP64 ones, the scarce unit, and select the same double bit for bit.
__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double okey_value(long long k)
{
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double min_t(double a, double b) { return okey(a) < okey(b) ? a : b; }
__device__ __forceinline__ float min_t(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double max_t(double a, double b) { return okey(a) < okey(b) ? b : a; }
__device__ __forceinline__ float max_t(float a, float b) { return fmaxf(a, b); }
// x >= 0 (either zero included) and x > 0 for non-NaN x, by the sign bit
__device__ __forceinline__ bool nonneg_t(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool nonneg_t(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool pos_t(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool pos_t(float x) { return x > 0.0f; }

// HLLC in vector form along the unit normal (nx,ny,nz): the tangential
// velocity rides along with the normal mass flux, so no explicit tangent
// basis is needed.  Davis wave speeds; contact speed from the jump conditions
// across the two outer waves.  Branch order: S_L >= 0 -> F_L; S* >= 0 -> F*_L;
// S_R > 0 -> F*_R; else F_R.
template <class T>
__device__ __forceinline__ void hllc_t(const FaceStateT<T> &L, const FaceStateT<T> &R, T nx, T ny, T nz, T gamma,
                                       T igm1, T F[5], WavesT<T> *wv = nullptr)
{
    const T ul = L.vx * nx + L.vy * ny + L.vz * nz;
    const T ur = R.vx * nx + R.vy * ny + R.vz * nz;
    const T cl = sqrt_t(gamma * L.P * L.irho), cr = sqrt_t(gamma * R.P * R.irho);
    const T El = L.P * igm1 + T(0.5) * L.rho * (L.vx * L.vx + L.vy * L.vy + L.vz * L.vz);
    const T Er = R.P * igm1 + T(0.5) * R.rho * (R.vx * R.vx + R.vy * R.vy + R.vz * R.vz);
    const T sl = min_t(ul - cl, ur - cr);
    const T sr = max_t(ul + cl, ur + cr);
    const T ml = L.rho * (sl - ul), mr = R.rho * (sr - ur);
    const T ss = (R.P - L.P + ul * ml - ur * mr) / (ml - mr);
    if (wv) *wv = WavesT<T>{sl, sr, ss, ul, ur};
    const bool left = nonneg_t(sl) || nonneg_t(ss);
    const bool star = !nonneg_t(sl) && (left || pos_t(sr));
    const FaceStateT<T> &K = left ? L : R;
    const T uk = left ? ul : ur;
    const T Ek = left ? El : Er;
    const T sk = left ? sl : sr;
    const T mk = K.rho * uk;
    // physical flux of side K
    F[0] = mk;
    F[1] = mk * K.vx + K.P * nx;
    F[2] = mk * K.vy + K.P * ny;
    F[3] = mk * K.vz + K.P * nz;
    F[4] = (Ek + K.P) * uk;
    if (star) {
        // U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, v_K + (S* - u_K) n, E_K/rho_K + (S* - u_K)(S* + P_K/(rho_K (S_K - u_K))))
        // With f = rho_K (S_K - u_K) / (S_K - S*), the energy term
        // f (S* - u_K) P_K / (rho_K (S_K - u_K)) equals (S* - u_K) P_K / (S_K - S*):
        // written that way the star state needs one division, and stays finite
        // where S_K rounds to u_K (a sound speed below the flow speed's ulp).
        const T rb = T(1) / (sk - ss);
        const T f = K.rho * (sk - uk) * rb;
        const T du = ss - uk;
        const T es = f * (Ek * K.irho + du * ss) + du * K.P * rb;
        F[0] += sk * (f - K.rho);
        F[1] += sk * (f * (K.vx + du * nx) - K.rho * K.vx);
        F[2] += sk * (f * (K.vy + du * ny) - K.rho * K.vy);
        F[3] += sk * (f * (K.vz + du * nz) - K.rho * K.vz);
        F[4] += sk * (es - Ek);
    }
}

// HLL with the same wave speeds: one intermediate state from the integral
// form of the conservation laws (no contact wave).
template <class T>
__device__ __forceinline__ void hll_t(const FaceStateT<T> &L, const FaceStateT<T> &R, T nx, T ny, T nz, T gamma,
                                      T igm1, T F[5], WavesT<T> *wv = nullptr)
{
    const T ul = L.vx * nx + L.vy * ny + L.vz * nz;
    const T ur = R.vx * nx + R.vy * ny + R.vz * nz;
    const T cl = sqrt_t(gamma * L.P * L.irho), cr = sqrt_t(gamma * R.P * R.irho);
    const T El = L.P * igm1 + T(0.5) * L.rho * (L.vx * L.vx + L.vy * L.vy + L.vz * L.vz);
    const T Er = R.P * igm1 + T(0.5) * R.rho * (R.vx * R.vx + R.vy * R.vy + R.vz * R.vz);
    const T sl = min_t(ul - cl, ur - cr);
    const T sr = max_t(ul + cl, ur + cr);
    if (wv) {
        // the contact speed of the same wave model, for the shock Mach number
        const T ss = (R.P - L.P + L.rho * ul * (sl - ul) - R.rho * ur * (sr - ur)) /
                     (L.rho * (sl - ul) - R.rho * (sr - ur));
        *wv = WavesT<T>{sl, sr, ss, ul, ur};
    }
    const T ml = L.rho * ul, mr = R.rho * ur;
    const T Fl[5] = {ml, ml * L.vx + L.P * nx, ml * L.vy + L.P * ny, ml * L.vz + L.P * nz, (El + L.P) * ul};
    const T Fr[5] = {mr, mr * R.vx + R.P * nx, mr * R.vy + R.P * ny, mr * R.vz + R.P * nz, (Er + R.P) * ur};
    if (sl >= T(0)) {
        for (int k = 0; k < 5; ++k) F[k] = Fl[k];
        return;
    }
    if (sr <= T(0)) {
        for (int k = 0; k < 5; ++k) F[k] = Fr[k];
        return;
    }
    const T Ul[5] = {L.rho, L.rho * L.vx, L.rho * L.vy, L.rho * L.vz, El};
    const T Ur[5] = {R.rho, R.rho * R.vx, R.rho * R.vy, R.rho * R.vz, Er};
    const T id = T(1) / (sr - sl);
    for (int k = 0; k < 5; ++k) F[k] = (sr * Fl[k] - sl * Fr[k] + sl * sr * (Ur[k] - Ul[k])) * id;
}

// Mach number of the shock that raises the pressure of either side to the
// star pressure (Rankine-Hugoniot: M^2 = 1 + k (P*/P - 1) with
// k = (gamma+1)/(2 gamma)), the larger of the two, 0 where neither side is
// compressed (Sec. 4.3).
template <class T>
__device__ __forceinline__ T shock_mach_t(T pl, T pr, T ps, T k)
{
    T m = T(0);
    if (ps > pl) m = max_t(m, sqrt_t(T(1) + k * (ps / pl - T(1))));
    if (ps > pr) m = max_t(m, sqrt_t(T(1) + k * (ps / pr - T(1))));
    return m;
}

// Flux of a passive charge rho a (the entropy column, Sec. 4.3) carried by
// the Riemann solution: HLLC takes a from the side of the contact times the
// mass flux fm; HLL averages rho a like any conserved column.
// The wave speeds are the solver's own (riemann_t with wv); the star pressure
// P* = P_L + rho_L (S_L - u_L)(S* - u_L) comes from the left wave's jump
// condition; kmach = (gamma+1)/(2 gamma).
template <class T>
__device__ __forceinline__ T passive_flux_t(int kind, const FaceStateT<T> &L, const FaceStateT<T> &R,
                                            const WavesT<T> &wv, T kmach, T rhoa_l, T rhoa_r, T fm, T &mach)
{
    const T sl = wv.sl, ss = wv.ss, sr = wv.sr, ul = wv.ul, ur = wv.ur;
    const T ps = L.P + L.rho * (sl - ul) * (ss - ul);
    mach = shock_mach_t<T>(L.P, R.P, ps, kmach);
    const T al = rhoa_l * L.irho, ar = rhoa_r * R.irho;
    if (kind == 1) {
        const T fl = L.rho * ul * al, fr = R.rho * ur * ar;
        if (sl >= T(0)) return fl;
        if (sr <= T(0)) return fr;
        return (sr * fl - sl * fr + sl * sr * (rhoa_r - rhoa_l)) / (sr - sl);
    }
    return fm * ((sl >= T(0) || ss >= T(0)) ? al : ar);
}

// The configured solver: 0 HLLC, 1 HLL.
template <class T>
__device__ __forceinline__ void riemann_t(int kind, const FaceStateT<T> &L, const FaceStateT<T> &R, T nx, T ny, T nz,
                                          T gamma, T igm1, T F[5], WavesT<T> *wv = nullptr)
{
    if (kind == 1) hll_t<T>(L, R, nx, ny, nz, gamma, igm1, F, wv);
    else hllc_t<T>(L, R, nx, ny, nz, gamma, igm1, F, wv);
}

// The same floors for a face state, also returning 1 / rho and the kinetic
// energy density of the result (for the pressure, without a second division).
template <class T>
__device__ __forceinline__ void apply_floor_ir_t(T W[5], T rho_floor, T eps_floor, T &ir, T &ke)
{
    if (!(W[0] >= rho_floor)) {
        W[0] = rho_floor;
        W[1] = W[2] = W[3] = T(0);
        W[4] = rho_floor * eps_floor;
        ir = T(1) / rho_floor;
        ke = T(0);
        return;
    }
    ir = T(1) / W[0];
    ke = T(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) * ir;
    if (!(W[4] - ke >= W[0] * eps_floor)) W[4] = W[0] * eps_floor + ke;
}

// Floors on density and specific internal energy (Sec. 4.1).  A state below
// the density floor is reset to the floor density at rest with the floor
// internal energy; otherwise only the internal energy is raised if needed.
// Returns true if the state changed (an untouched state is left bit for bit).
template <class T>
__device__ __forceinline__ bool apply_floor_t(T W[5], T rho_floor, T eps_floor)
{
    if (!(W[0] >= rho_floor)) {
        W[0] = rho_floor;
        W[1] = W[2] = W[3] = T(0);
        W[4] = rho_floor * eps_floor;
        return true;
    }
    const T ke = T(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0];
    if (!(W[4] - ke >= W[0] * eps_floor)) {
        W[4] = W[0] * eps_floor + ke;
        return true;
    }
    return false;
}

}  // namespace mm
