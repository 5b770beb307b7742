// Device code of libamr, templated on the storage type T (float or double),
// the dimension D and the patch size N. Included by amr_f32.cu and amr_f64.cu.
//
// Every floating-point expression is written in a fixed evaluation order. The
// FP64 unit is compiled with -fmad=false, so each operation rounds once and the
// FP64 path reproduces an IEEE evaluation of the same formulas on the host.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <type_traits>
#include <cstdint>
#include "amr_internal.h"
#include "amr.h"

namespace amr {

// ---------------------------------------------------------------------------
// arithmetic helpers: FP64 uses IEEE division and square root; FP32 uses the
// fast approximate forms (the FP32 path is compared by tolerance, not bits)
// ---------------------------------------------------------------------------
template <typename T> struct Num;
template <> struct Num<double> {
    __device__ __forceinline__ static double div(double a, double b) { return a / b; }
    __device__ __forceinline__ static double sqr(double a) { return sqrt(a); }
};
template <> struct Num<float> {
    __device__ __forceinline__ static float div(float a, float b) { return __fdividef(a, b); }
    __device__ __forceinline__ static float sqr(float a) { return sqrtf(a); }
};

template <typename T, int N> struct PatchShape {
    static constexpr int S = N + 2 * G;                  // cells per slot side
    static constexpr int PER32 = 32 / (int)sizeof(T);    // elements per 32-byte sector
    static constexpr int XP = (PER32 - G % PER32) % PER32;   // pad before the first ghost of a row
    static constexpr int SX = (XP + S + 7) / 8 * 8;      // padded x pitch
    static_assert((XP + G) % PER32 == 0, "interior rows start on a 32-byte boundary");
};

__device__ __forceinline__ int floordiv(int a, int b) {
    int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

__device__ __forceinline__ long long slot_index(const Grid& g, int slot, int v, int sz, int sy, int sx) {
    return (long long)slot * g.patch_elems + (long long)v * g.slot_elems +
           ((long long)sz * g.SY + sy) * g.SX + sx + g.XP;
}

// 16-byte vector of VE consecutive elements (FP32: 4, FP64: 2) at an aligned address
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int VE = 4;
    __device__ __forceinline__ static void load(const float* p, float (&o)[4]) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
    __device__ __forceinline__ static void store(float* p, const float (&o)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct Vec16<double> {
    static constexpr int VE = 2;
    __device__ __forceinline__ static void load(const double* p, double (&o)[2]) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        o[0] = t.x; o[1] = t.y;
    }
    __device__ __forceinline__ static void store(double* p, const double (&o)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};

// slot coordinate of local index l in an active (d < D) or inactive dimension
template <int D>
__device__ __forceinline__ int sc(int d, int l) { return d < D ? l + G : 0; }

// ---------------------------------------------------------------------------
// Euler primitives (Sec. 3.1, Eqs. 4-6, R = 1): u = m / rho,
// p = (gamma - 1)(E - rho |u|^2 / 2), T = p / rho
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void primitives(const T* U, T gm1, T& rho, T* u, T& p, T& Tt) {
    rho = U[0];
    T usq = T(0);
    if constexpr (sizeof(T) == 4) {                  // FP32: one reciprocal for the D + 1 quotients
        const float r = __fdividef(1.0f, rho);
#pragma unroll
        for (int d = 0; d < D; ++d) u[d] = U[1 + d] * r;
        usq = u[0] * u[0];
#pragma unroll
        for (int d = 1; d < D; ++d) usq = usq + u[d] * u[d];
        p = gm1 * (U[D + 1] - T(0.5) * rho * usq);
        Tt = p * r;
        return;
    }
#pragma unroll
    for (int d = 0; d < D; ++d) u[d] = Num<T>::div(U[1 + d], rho);
    usq = u[0] * u[0];
#pragma unroll
    for (int d = 1; d < D; ++d) usq = usq + u[d] * u[d];
    p = gm1 * (U[D + 1] - T(0.5) * rho * usq);
    Tt = Num<T>::div(p, rho);
}

template <int D>
__device__ __forceinline__ double pressure_d(const double* U, double gm1) {
    double rho = U[0];
    double u[3];
#pragma unroll
    for (int d = 0; d < D; ++d) u[d] = U[1 + d] / rho;
    double usq = u[0] * u[0];
#pragma unroll
    for (int d = 1; d < D; ++d) usq = usq + u[d] * u[d];
    return gm1 * (U[D + 1] - 0.5 * rho * usq);
}

// ---------------------------------------------------------------------------
// WENO5-JS nodal mid-point interpolation at x_{i+1/2} from nodes i-2..i+2
// (Sec. 3.2): quadratic candidates, linear weights (1, 10, 5)/16, Jiang-Shu
// smoothness indicators, alpha_k = d_k / (eps + beta_k)^2, eps = 1e-6
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e) {
    const T q0 = (T(3) * a - T(10) * b + T(15) * c) * T(0.125);
    const T q1 = (-b + T(6) * c + T(3) * d) * T(0.125);
    const T q2 = (T(3) * c + T(6) * d - e) * T(0.125);
    const T t0 = a - T(2) * b + c;
    const T s0 = a - T(4) * b + T(3) * c;
    const T t1 = b - T(2) * c + d;
    const T s1 = b - d;
    const T t2 = c - T(2) * d + e;
    const T s2 = T(3) * c - T(4) * d + e;
    const T c1312 = T(13.0 / 12.0);
    const T b0 = c1312 * (t0 * t0) + T(0.25) * (s0 * s0);
    const T b1 = c1312 * (t1 * t1) + T(0.25) * (s1 * s1);
    const T b2 = c1312 * (t2 * t2) + T(0.25) * (s2 * s2);
    const T e0 = T(1.0e-6) + b0;
    const T e1 = T(1.0e-6) + b1;
    const T e2 = T(1.0e-6) + b2;
    const T a0 = Num<T>::div(T(0.0625), e0 * e0);
    const T a1 = Num<T>::div(T(0.625), e1 * e1);
    const T a2 = Num<T>::div(T(0.3125), e2 * e2);
    return Num<T>::div(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

// FP32: left- (nodes 0..4) and right-biased (nodes 5..1) WENO5-JS values of one
// face together; the right stencil is the left one mirrored, so two candidate
// values and two smoothness terms are shared between them. Same formulas as
// weno5. FAST: the normalised weights are unchanged when every alpha_k is
// multiplied by e0^2 e1^2 e2^2, which leaves a single division, exact up to
// rounding while no product overflows: checked on the division's operands, a
// finite numerator and a denominator below 2^126, the range of the fast
// division (the denominator is at least 0.0625 eps^4, far above 2^-126). ok
// is cleared otherwise, and the caller evaluates the face again without FAST;
// else three divisions.
__device__ __forceinline__ bool weights_in_range(float num, float den) {
    return fabsf(num) < 1.0e37f && den < 1.0e37f;
}
template <bool FAST>
__device__ __forceinline__ void weno5_pair(float v0, float v1, float v2, float v3, float v4, float v5, float& left,
                                           float& right, bool& ok) {
    const float c1312 = 13.0f / 12.0f;
    const float qA = (-v1 + 6.0f * v2 + 3.0f * v3) * 0.125f;   // left q1 = right q2
    const float qB = (3.0f * v2 + 6.0f * v3 - v4) * 0.125f;    // left q2 = right q1
    const float tA = v1 - 2.0f * v2 + v3, tB = v2 - 2.0f * v3 + v4;
    const float cA = c1312 * (tA * tA), cB = c1312 * (tB * tB);
    auto combine = [&ok](float q0, float q1, float q2, float b0, float b1, float b2) {
        const float e0 = 1.0e-6f + b0, e1 = 1.0e-6f + b1, e2 = 1.0e-6f + b2;
        const float s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
        if constexpr (FAST) {
            const float m0 = 0.0625f * (s1 * s2), m1 = 0.625f * (s0 * s2), m2 = 0.3125f * (s0 * s1);
            const float num = m0 * q0 + m1 * q1 + m2 * q2, den = m0 + m1 + m2;
            ok = ok && weights_in_range(num, den);
            return __fdividef(num, den);
        } else {
            const float a0 = __fdividef(0.0625f, s0), a1 = __fdividef(0.625f, s1), a2 = __fdividef(0.3125f, s2);
            return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
        }
    };
    {   // left: a = v0, b = v1, c = v2, d = v3, e = v4
        const float q0 = (3.0f * v0 - 10.0f * v1 + 15.0f * v2) * 0.125f;
        const float t0 = v0 - 2.0f * v1 + v2, s0 = v0 - 4.0f * v1 + 3.0f * v2;
        const float s1 = v1 - v3, s2 = 3.0f * v2 - 4.0f * v3 + v4;
        left = combine(q0, qA, qB, c1312 * (t0 * t0) + 0.25f * (s0 * s0), cA + 0.25f * (s1 * s1),
                       cB + 0.25f * (s2 * s2));
    }
    {   // right: a = v5, b = v4, c = v3, d = v2, e = v1
        const float q0 = (3.0f * v5 - 10.0f * v4 + 15.0f * v3) * 0.125f;
        const float t0 = v5 - 2.0f * v4 + v3, s0 = v5 - 4.0f * v4 + 3.0f * v3;
        const float s1 = v4 - v2, s2 = 3.0f * v3 - 4.0f * v2 + v1;
        right = combine(q0, qB, qA, c1312 * (t0 * t0) + 0.25f * (s0 * s0), cB + 0.25f * (s1 * s1),
                        cA + 0.25f * (s2 * s2));
    }
}

// ---------------------------------------------------------------------------
// Packed FP32 (Blackwell f32x2): two independent lanes per instruction.
// ---------------------------------------------------------------------------
struct F2 {
    float2 v;
};
__device__ __forceinline__ F2 f2(float x, float y) { return {make_float2(x, y)}; }
__device__ __forceinline__ F2 f2s(float s) { return {make_float2(s, s)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, float s) { return {__fmul2_rn(a.v, make_float2(s, s))}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, float s, F2 c) { return {__ffma2_rn(a.v, make_float2(s, s), c.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
// approximate reciprocal (PTX rcp.approx, about 1 ulp; operands here are
// normal numbers) of both lanes
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ F2 rcp2(F2 a) { return f2(rcp_approx(a.v.x), rcp_approx(a.v.y)); }

// the weights of weno5_pair<true> on both lanes, from candidates q and
// smoothness indicators b given as 4 beta_k (with eps scaled alike: the
// normalised weights are unchanged) and without the common factor 1/16 of the
// linear weights (1, 10, 5) / 16; LIN: q1 and q2 come multiplied by their
// linear weights 10 and 5. ok is cleared when either lane's division is out
// of range.
template <bool LIN>
__device__ __forceinline__ F2 weno5_combine_x2(F2 q0, F2 q1, F2 q2, F2 b0, F2 b1, F2 b2, bool& ok) {
    const F2 eps = f2s(4.0e-6f);
    const F2 e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
    const F2 s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
    const F2 p12 = s1 * s2, p02 = s0 * s2, p01 = s0 * s1;
    F2 num, den;
    if constexpr (LIN) {
        num = fma2(p01, q2, fma2(p02, q1, p12 * q0));
        den = fma2(p01, 5.0f, fma2(p02, 10.0f, p12));
    } else {
        const F2 m1 = p02 * 10.0f, m2 = p01 * 5.0f;
        num = fma2(m2, q2, fma2(m1, q1, p12 * q0));
        den = p12 + m1 + m2;
    }
    ok = ok && weights_in_range(num.v.x, den.v.x) && weights_in_range(num.v.y, den.v.y);
    return num * rcp2(den);
}

// weno5_pair<FAST> on two characteristic fields at once (lane x and lane y):
// the same candidates, smoothness indicators and single-division weights,
// evaluated with packed instructions; ok is cleared when a weight product of
// either lane would leave the FP32 range
__device__ __forceinline__ void weno5_pair_x2(F2 v0, F2 v1, F2 v2, F2 v3, F2 v4, F2 v5, F2& left, F2& right,
                                              bool& ok) {
    const float c133 = 13.0f / 3.0f;                                      // 4 beta = 13/3 t^2 + s^2
    const F2 qA = fma2(v3, 0.375f, fma2(v2, 0.75f, v1 * -0.125f));     // left q1 = right q2
    const F2 qB = fma2(v4, -0.125f, fma2(v3, 0.75f, v2 * 0.375f));     // left q2 = right q1
    const F2 tA = fma2(v2, -2.0f, v1 + v3), tB = fma2(v3, -2.0f, v2 + v4);
    const F2 cA = tA * (tA * c133), cB = tB * (tB * c133);
    auto beta4 = [c133](F2 t, F2 s) { return fma2(t, t * c133, s * s); };
    {   // left: a = v0, b = v1, c = v2, d = v3, e = v4
        const F2 q0 = fma2(v2, 1.875f, fma2(v1, -1.25f, v0 * 0.375f));
        const F2 t0 = fma2(v1, -2.0f, v0 + v2), s0 = fma2(v1, -4.0f, fma2(v2, 3.0f, v0));
        const F2 s1 = v1 - v3, s2 = fma2(v3, -4.0f, fma2(v2, 3.0f, v4));
        left = weno5_combine_x2<false>(q0, qA, qB, beta4(t0, s0), fma2(s1, s1, cA), fma2(s2, s2, cB), ok);
    }
    {   // right: a = v5, b = v4, c = v3, d = v2, e = v1
        const F2 q0 = fma2(v3, 1.875f, fma2(v4, -1.25f, v5 * 0.375f));
        const F2 t0 = fma2(v4, -2.0f, v5 + v3), s0 = fma2(v4, -4.0f, fma2(v3, 3.0f, v5));
        const F2 s1 = v4 - v2, s2 = fma2(v2, -4.0f, fma2(v3, 3.0f, v1));
        right = weno5_combine_x2<false>(q0, qB, qA, beta4(t0, s0), fma2(s1, s1, cB), fma2(s2, s2, cA), ok);
    }
}

// weno5 (single-division weights) of two stencils a..e at once, one per lane:
// used for the left (nodes 0..4) and right (nodes 5..1) values of one field
__device__ __forceinline__ F2 weno5_x2(F2 a, F2 b, F2 c, F2 d, F2 e, bool& ok) {
    const float c133 = 13.0f / 3.0f;
    const F2 q0 = fma2(c, 1.875f, fma2(b, -1.25f, a * 0.375f));
    const F2 q1 = fma2(d, 3.75f, fma2(c, 7.5f, b * -1.25f));          // 10 q1
    const F2 q2 = fma2(e, -0.625f, fma2(d, 3.75f, c * 1.875f));       // 5 q2
    const F2 t0 = fma2(b, -2.0f, a + c), s0 = fma2(b, -4.0f, fma2(c, 3.0f, a));
    const F2 t1 = fma2(c, -2.0f, b + d), s1 = b - d;
    const F2 t2 = fma2(d, -2.0f, c + e), s2 = fma2(d, -4.0f, fma2(c, 3.0f, e));
    auto beta4 = [c133](F2 t, F2 s) { return fma2(t, t * c133, s * s); };
    return weno5_combine_x2<true>(q0, q1, q2, beta4(t0, s0), beta4(t1, s1), beta4(t2, s2), ok);
}
// left and right WENO values of one field with nodes v[0..5], as one packed call
__device__ __forceinline__ void weno5_lr_x2(float v0, float v1, float v2, float v3, float v4, float v5, float& left,
                                            float& right, bool& ok) {
    const F2 r = weno5_x2(f2(v0, v5), f2(v1, v4), f2(v2, v3), f2(v3, v2), f2(v4, v1), ok);
    left = r.v.x;
    right = r.v.y;
}

// left and right values of one characteristic field; FP32 see weno5_pair
template <typename T, bool FAST>
__device__ __forceinline__ void weno5_lr(const T (&w)[6], T& left, T& right, bool& ok) {
    if constexpr (sizeof(T) == 4) {
        weno5_pair<FAST>(w[0], w[1], w[2], w[3], w[4], w[5], left, right, ok);
    } else {
        left = weno5(w[0], w[1], w[2], w[3], w[4]);
        right = weno5(w[5], w[4], w[3], w[2], w[1]);
    }
}

// ---------------------------------------------------------------------------
// Face flux between pencil nodes 2 and 3 (Sec. 3.2, Eqs. 10-12).
// Pencil node k holds (p, un, ut[NT], T). Frozen state: pbar, Tbar means of
// nodes 2, 3; rhobar = pbar / Tbar; cbar = sqrt(gamma Tbar); z = rhobar cbar;
// kappa = (gamma-1) / (gamma rhobar). Characteristic fields of the primitive
// system in (p, u, T): w1 = p - z un, w2 = T - kappa p, w_t = ut, w5 = p + z un.
// Left/right WENO5, inverse transform, first-order fallback if p or T is not
// positive, Rusanov flux with S = max(c + |un|), or (flux = AMR_FLUX_HLLC)
// the HLLC flux of the same states: wave-speed bounds S_L = min(un - c),
// S_R = max(un + c) over the sides, contact speed S*, star states and the
// four-way choice by the signs of S_L, S*, S_R. Output in pencil order (mass,
// normal momentum, tangential momenta, energy).
// ---------------------------------------------------------------------------
template <typename T, int NT, int FLUX>
__device__ __forceinline__ void face_flux(const T (&p)[6], const T (&un)[6], const T (&ut)[NT > 0 ? NT : 1][6],
                                          const T (&Tt)[6], T gamma, T gm1, T (&F)[NT + 3]) {
    constexpr int NF = NT + 3;
    const T pbar = T(0.5) * (p[2] + p[3]);
    const T Tbar = T(0.5) * (Tt[2] + Tt[3]);
    const T rbar = Num<T>::div(pbar, Tbar);
    const T cbar = Num<T>::sqr(gamma * Tbar);
    const T z = rbar * cbar;
    const T kap = Num<T>::div(gm1, gamma * rbar);
    T wl[NF], wr[NF];
    // FP32: every field with the single-division weights, and the whole face
    // again with three divisions in the rare case one of them was out of range
    auto interpolate = [&](auto fast) {
        constexpr bool FAST = decltype(fast)::value;
        bool ok = true;
        T w[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = p[k] - z * un[k];
        weno5_lr<T, FAST>(w, wl[0], wr[0], ok);
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = Tt[k] - kap * p[k];
        weno5_lr<T, FAST>(w, wl[1], wr[1], ok);
#pragma unroll
        for (int j = 0; j < NT; ++j) weno5_lr<T, FAST>(ut[j], wl[2 + j], wr[2 + j], ok);
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = p[k] + z * un[k];
        weno5_lr<T, FAST>(w, wl[NF - 1], wr[NF - 1], ok);
        return ok;
    };
    if (!interpolate(std::true_type{})) {
        if constexpr (sizeof(T) == 4) interpolate(std::false_type{});
    }
    const T z2 = T(2) * z;
    T pL = T(0.5) * (wl[0] + wl[NF - 1]);
    T unL = Num<T>::div(wl[NF - 1] - wl[0], z2);
    T TL = wl[1] + kap * pL;
    T pR = T(0.5) * (wr[0] + wr[NF - 1]);
    T unR = Num<T>::div(wr[NF - 1] - wr[0], z2);
    T TR = wr[1] + kap * pR;
    T utL[NT > 0 ? NT : 1], utR[NT > 0 ? NT : 1];
#pragma unroll
    for (int j = 0; j < NT; ++j) { utL[j] = wl[2 + j]; utR[j] = wr[2 + j]; }
    const bool bad = !(pL > T(0)) || !(TL > T(0)) || !(pR > T(0)) || !(TR > T(0));
    if (bad) {
        pL = p[2]; unL = un[2]; TL = Tt[2];
        pR = p[3]; unR = un[3]; TR = Tt[3];
#pragma unroll
        for (int j = 0; j < NT; ++j) { utL[j] = ut[j][2]; utR[j] = ut[j][3]; }
    }
    // conserved states and Euler fluxes at both sides
    T UL[NF], FL[NF], UR[NF], FR[NF];
    T sL, sR;
    T rhoS[2], ES[2], cS[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const T ps = side ? pR : pL;
        const T uns = side ? unR : unL;
        const T Ts = side ? TR : TL;
        const T rho = Num<T>::div(ps, Ts);
        const T c = Num<T>::sqr(gamma * Ts);
        T usq = uns * uns;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const T v = side ? utR[j] : utL[j];
            usq = usq + v * v;
        }
        const T E = Num<T>::div(ps, gm1) + T(0.5) * rho * usq;
        const T mn = rho * uns;
        T* Uo = side ? UR : UL;
        T* Fo = side ? FR : FL;
        Uo[0] = rho;
        Uo[1] = mn;
        Fo[0] = mn;
        Fo[1] = mn * uns + ps;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const T v = side ? utR[j] : utL[j];
            Uo[2 + j] = rho * v;
            Fo[2 + j] = mn * v;
        }
        Uo[NF - 1] = E;
        Fo[NF - 1] = (E + ps) * uns;
        const T s = c + fabs(uns);
        if (side) sR = s; else sL = s;
        rhoS[side] = rho;
        ES[side] = E;
        cS[side] = c;
    }
    if constexpr (FLUX == AMR_FLUX_HLLC) {
        const T wL = fmin(unL - cS[0], unR - cS[1]);
        const T wR = fmax(unL + cS[0], unR + cS[1]);
        const T aL = rhoS[0] * (wL - unL);
        const T aR = rhoS[1] * (wR - unR);
        const T sM = Num<T>::div(pR - pL + aL * unL - aR * unR, aL - aR);
        if (wL >= T(0)) {                                  // F_L, F*_L (S* >= 0), F*_R (S_R > 0), F_R
#pragma unroll
            for (int v = 0; v < NF; ++v) F[v] = FL[v];
        } else if (!(sM >= T(0)) && !(wR > T(0))) {
#pragma unroll
            for (int v = 0; v < NF; ++v) F[v] = FR[v];
        } else {
            const bool left = sM >= T(0);               // the star state on the contact's upwind side
            const T a = left ? aL : aR, w = left ? wL : wR, un_s = left ? unL : unR, p_s = left ? pL : pR;
            const T* Uo = left ? UL : UR;
            const T* Fo = left ? FL : FR;
            const T f = Num<T>::div(a, w - sM);
            T Us[NF];
            Us[0] = f;
            Us[1] = f * sM;
#pragma unroll
            for (int j = 0; j < NT; ++j) Us[2 + j] = f * (left ? utL[j] : utR[j]);
            Us[NF - 1] = f * (Num<T>::div(ES[left ? 0 : 1], rhoS[left ? 0 : 1]) + (sM - un_s) * (sM + Num<T>::div(p_s, a)));
#pragma unroll
            for (int v = 0; v < NF; ++v) F[v] = Fo[v] + w * (Us[v] - Uo[v]);
        }
        return;
    }
    const T hS = T(0.5) * fmax(sR, sL);
#pragma unroll
    for (int v = 0; v < NF; ++v) F[v] = T(0.5) * (FR[v] + FL[v]) - hS * (UR[v] - UL[v]);
}

// ---------------------------------------------------------------------------
// FP32 Rusanov face flux with packed arithmetic: the same steps as face_flux
// (frozen state, characteristic fields, WENO5-JS left/right, inverse
// transform, first-order fallback, Rusanov flux). The characteristic fields
// go through WENO in pairs, (w1, w5) and (w2, w_t1) (w_t2 alone in 3D, w2
// alone in 1D), and the two face sides' conserved states and fluxes are
// formed as pairs (left, right).
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void face_flux_x2(const float (&p)[6], const float (&un)[6],
                                             const float (&ut)[NT > 0 ? NT : 1][6], const float (&Tt)[6],
                                             float gamma, float gm1, float (&F)[NT + 3]) {
    constexpr int NF = NT + 3;
    const float pbar = 0.5f * (p[2] + p[3]);
    const float Tbar = 0.5f * (Tt[2] + Tt[3]);
    const float rbar = __fdividef(pbar, Tbar);
    const float cbar = sqrtf(gamma * Tbar);
    const float z = rbar * cbar;
    const float kap = __fdividef(gm1, gamma * rbar);
    float wl[NF], wr[NF];
    bool ok = true;
    {
        F2 a[6], b[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            a[k] = f2(fmaf(-z, un[k], p[k]), fmaf(z, un[k], p[k]));                 // (w1, w5)
            b[k] = f2(fmaf(-kap, p[k], Tt[k]), NT >= 1 ? ut[0][k] : 0.0f);          // (w2, w_t1)
        }
        F2 L, R;
        weno5_pair_x2(a[0], a[1], a[2], a[3], a[4], a[5], L, R, ok);
        wl[0] = L.v.x; wl[NF - 1] = L.v.y; wr[0] = R.v.x; wr[NF - 1] = R.v.y;
        if constexpr (NT >= 1) {
            weno5_pair_x2(b[0], b[1], b[2], b[3], b[4], b[5], L, R, ok);
            wl[1] = L.v.x; wl[2] = L.v.y; wr[1] = R.v.x; wr[2] = R.v.y;
        } else {
            weno5_lr_x2(b[0].v.x, b[1].v.x, b[2].v.x, b[3].v.x, b[4].v.x, b[5].v.x, wl[1], wr[1], ok);
        }
        if constexpr (NT == 2) weno5_lr_x2(ut[1][0], ut[1][1], ut[1][2], ut[1][3], ut[1][4], ut[1][5], wl[3], wr[3], ok);
    }
    if (!ok) {          // a weight product out of range: every field again with three divisions
        float w[6];
        bool ok2 = true;
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = p[k] - z * un[k];
        weno5_pair<false>(w[0], w[1], w[2], w[3], w[4], w[5], wl[0], wr[0], ok2);
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = Tt[k] - kap * p[k];
        weno5_pair<false>(w[0], w[1], w[2], w[3], w[4], w[5], wl[1], wr[1], ok2);
#pragma unroll
        for (int j = 0; j < NT; ++j)
            weno5_pair<false>(ut[j][0], ut[j][1], ut[j][2], ut[j][3], ut[j][4], ut[j][5], wl[2 + j], wr[2 + j], ok2);
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = p[k] + z * un[k];
        weno5_pair<false>(w[0], w[1], w[2], w[3], w[4], w[5], wl[NF - 1], wr[NF - 1], ok2);
    }
    // inverse transform of both sides, as (left, right) pairs
    const float i2z = __fdividef(0.5f, z);
    F2 P = f2(0.5f * (wl[0] + wl[NF - 1]), 0.5f * (wr[0] + wr[NF - 1]));
    F2 UN = f2((wl[NF - 1] - wl[0]) * i2z, (wr[NF - 1] - wr[0]) * i2z);
    F2 TT = fma2(P, kap, f2(wl[1], wr[1]));
    F2 UT[NT > 0 ? NT : 1];
#pragma unroll
    for (int j = 0; j < NT; ++j) UT[j] = f2(wl[2 + j], wr[2 + j]);
    const bool bad = !(P.v.x > 0.f) || !(TT.v.x > 0.f) || !(P.v.y > 0.f) || !(TT.v.y > 0.f);
    if (bad) {
        P = f2(p[2], p[3]);
        UN = f2(un[2], un[3]);
        TT = f2(Tt[2], Tt[3]);
#pragma unroll
        for (int j = 0; j < NT; ++j) UT[j] = f2(ut[j][2], ut[j][3]);
    }
    // conserved states and Euler fluxes of both sides
    const F2 RHO = f2(__fdividef(P.v.x, TT.v.x), __fdividef(P.v.y, TT.v.y));
    const F2 GT = TT * gamma;
    const F2 C = f2(sqrtf(GT.v.x), sqrtf(GT.v.y));
    F2 usq = UN * UN;
#pragma unroll
    for (int j = 0; j < NT; ++j) usq = fma2(UT[j], UT[j], usq);
    const F2 E = fma2(RHO * 0.5f, usq, P * (1.0f / gm1));
    const F2 MN = RHO * UN;
    F2 U[NF], FF[NF];
    U[0] = RHO;
    U[1] = MN;
    FF[0] = MN;
    FF[1] = fma2(MN, UN, P);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        U[2 + j] = RHO * UT[j];
        FF[2 + j] = MN * UT[j];
    }
    U[NF - 1] = E;
    FF[NF - 1] = (E + P) * UN;
    const float hS = 0.5f * fmaxf(C.v.y + fabsf(UN.v.y), C.v.x + fabsf(UN.v.x));
#pragma unroll
    for (int v = 0; v < NF; ++v) F[v] = 0.5f * (FF[v].v.y + FF[v].v.x) - hS * (U[v].v.y - U[v].v.x);
}

// ---------------------------------------------------------------------------
// Shock-free face flux (Sec. 3.2, Eq. 8 read as the edge value from node
// values): p, u_n, u_t, T at the face from pencil nodes 1..4 (cells i-1 ..
// i+2) by (9 (phi_i + phi_{i+1}) - (phi_{i-1} + phi_{i+2})) / 16; if p or T is
// not positive there, the mean of nodes 2 and 3. The flux is the Euler flux of
// that one edge state (no dissipation). Output in pencil order.
// ---------------------------------------------------------------------------
// OFF shifts the four nodes by -1, 0 or +1 (the faces i - 1/2, i + 1/2,
// i + 3/2 of the hybrid flux below).
template <typename T, int NT, int OFF = 0>
__device__ __forceinline__ void central_flux(const T (&p)[6], const T (&un)[6], const T (&ut)[NT > 0 ? NT : 1][6],
                                             const T (&Tt)[6], T gm1, T (&F)[NT + 3]) {
    constexpr int NF = NT + 3;
    constexpr int A = 1 + OFF, B = 2 + OFF, C = 3 + OFF, D = 4 + OFF;
    auto mid = [](const T (&v)[6]) { return (T(9) * (v[B] + v[C]) - (v[A] + v[D])) * T(0.0625); };
    T pf = mid(p), unf = mid(un), Tf = mid(Tt);
    T utf[NT > 0 ? NT : 1];
#pragma unroll
    for (int j = 0; j < NT; ++j) utf[j] = mid(ut[j]);
    if (!(pf > T(0)) || !(Tf > T(0))) {
        pf = T(0.5) * (p[B] + p[C]);
        unf = T(0.5) * (un[B] + un[C]);
        Tf = T(0.5) * (Tt[B] + Tt[C]);
#pragma unroll
        for (int j = 0; j < NT; ++j) utf[j] = T(0.5) * (ut[j][B] + ut[j][C]);
    }
    const T rho = Num<T>::div(pf, Tf);
    T usq = unf * unf;
#pragma unroll
    for (int j = 0; j < NT; ++j) usq = usq + utf[j] * utf[j];
    const T E = Num<T>::div(pf, gm1) + T(0.5) * rho * usq;
    const T mn = rho * unf;
    F[0] = mn;
    F[1] = mn * unf + pf;
#pragma unroll
    for (int j = 0; j < NT; ++j) F[2 + j] = mn * utf[j];
    F[NF - 1] = (E + pf) * unf;
}

// ---------------------------------------------------------------------------
// Hybrid face value between pencil nodes 2 and 3 (Sec. 3.2: central schemes
// for shock-free flow, characteristic WENO5 + Rusanov for shocks; the choice
// face by face is an extension). Shock sensor: at nodes 1..4 and for phi in
// (rho = p / T, p), |phi_{k+1} - phi_{k-1}| > theta (phi_{k+1} + 2 phi_k +
// phi_{k-1}). Quiet: the central scheme's conservative face value
// (26 F_c(i+1/2) - F_c(i-1/2) - F_c(i+3/2)) / 24 (Eq. 9) from the central
// fluxes of nodes 1..4, 0..3 and 2..5; else the WENO5 + Rusanov flux.
// ---------------------------------------------------------------------------
template <typename T, int NT>
__device__ __forceinline__ void hybrid_flux(const T (&p)[6], const T (&un)[6], const T (&ut)[NT > 0 ? NT : 1][6],
                                            const T (&Tt)[6], T gamma, T gm1, T theta, T (&F)[NT + 3]) {
    constexpr int NF = NT + 3;
    T rho[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rho[k] = Num<T>::div(p[k], Tt[k]);
    bool shock = false;
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        shock = shock || fabs(rho[k + 1] - rho[k - 1]) > theta * (rho[k + 1] + T(2) * rho[k] + rho[k - 1]);
        shock = shock || fabs(p[k + 1] - p[k - 1]) > theta * (p[k + 1] + T(2) * p[k] + p[k - 1]);
    }
    if (shock) {
        if constexpr (sizeof(T) == 4) face_flux_x2<NT>(p, un, ut, Tt, gamma, gm1, F);
        else face_flux<T, NT, AMR_FLUX_RUSANOV>(p, un, ut, Tt, gamma, gm1, F);
        return;
    }
    T Fl[NF], Fm[NF], Fh[NF];
    central_flux<T, NT, -1>(p, un, ut, Tt, gm1, Fl);
    central_flux<T, NT, 0>(p, un, ut, Tt, gm1, Fm);
    central_flux<T, NT, 1>(p, un, ut, Tt, gm1, Fh);
#pragma unroll
    for (int v = 0; v < NF; ++v) {
        const T gsum = T(26) * Fm[v] - Fl[v] - Fh[v];
        F[v] = sizeof(T) == 4 ? gsum * T(1.0 / 24.0) : gsum / T(24);
    }
}

// Metadata of one patch staged in shared memory by the CTA that serves it:
// level, coordinates, its 27-entry neighbour table and its parent's.
struct PatchMeta {
    int slot, lev, par;
    int c[3];
    int nbr[NBR];
    int pnbr[NBR];
};

__device__ __forceinline__ void load_meta(const Grid& g, int slot, PatchMeta& m) {
    const int t = threadIdx.x;
    if (t == 0) {
        m.slot = slot;
        m.lev = g.level[slot];
        m.par = g.parent[slot];
        m.c[0] = g.coord[slot * 3];
        m.c[1] = g.coord[slot * 3 + 1];
        m.c[2] = g.coord[slot * 3 + 2];
    }
    if (t < NBR) m.nbr[t] = g.nbr[slot * NBR + t];
    if (t >= 32 && t < 32 + NBR) {
        const int par = g.parent[slot];
        m.pnbr[t - 32] = par >= 0 ? g.nbr[par * NBR + t - 32] : -1;
    }
    __syncthreads();
}

// the same, by one warp into its own copy (no CTA barrier)
__device__ __forceinline__ void load_meta_warp(const Grid& g, int slot, PatchMeta& m) {
    const int lane = threadIdx.x & 31;
    const int par = g.parent[slot];
    if (lane == 0) {
        m.slot = slot;
        m.lev = g.level[slot];
        m.par = par;
        m.c[0] = g.coord[slot * 3];
        m.c[1] = g.coord[slot * 3 + 1];
        m.c[2] = g.coord[slot * 3 + 2];
    }
    if (lane < NBR) {
        m.nbr[lane] = g.nbr[slot * NBR + lane];
        m.pnbr[lane] = par >= 0 ? g.nbr[par * NBR + lane] : -1;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Limited-linear prolongation of the conserved variables at fine local cell l
// of a patch (slot, level lev, coords c): coarse cell C = G // 2 in the
// parent's Moore neighbourhood (guaranteed by R2), minmod slopes of the
// neighbouring differences (tie: first argument U_{C+1} - U_C), child value
// U_C + sum_d (+-1/4) s_d, dims in order; U_C for every child of C if any
// child has rho <= 0 or p <= 0.
// ---------------------------------------------------------------------------
// NBR_READS (the ghost fill): C +- e_d outside Q is read from Q's same-level
// neighbour when it exists, as a stage leaves that face ghost of Q unfilled;
// otherwise (new patches in a regrid, which may create that neighbour in the
// same launch) from Q's ghost cells, filled before the mesh changed.
// The coarse cell C of fine local cell l: returns Q, the patch that holds C
// (from the parent's neighbour table; -1 if there is none), and sets C's
// local coordinates Lc in Q and the child index s of l (bit d: the upper half
// along d)
template <int D, int N>
__device__ __forceinline__ int prolong_locate(const PatchMeta& m, const int* l, int* Lc, int* s) {
    const int* c = m.c;
    int oc[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Lc[d] = 0;
        s[d] = 0;
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int Gd = c[d] * N + l[d];
        const int Gc = Gd >> 1;                 // floor (arithmetic shift)
        s[d] = Gd - 2 * Gc;
        const int PC = c[d] >> 1;
        oc[d] = floordiv(Gc, N) - PC;
        Lc[d] = Gc - (PC + oc[d]) * N;
    }
    return m.par >= 0 ? m.pnbr[(oc[2] + 1) * 9 + (oc[1] + 1) * 3 + (oc[0] + 1)] : -1;
}

// U_C and the minmod slopes of coarse cell Lc of Q (NBR_READS: see below)
template <typename T, int D, int N, bool NBR_READS>
__device__ __forceinline__ void prolong_slopes(const Grid& g, const T* U, int Q, const int* Lc, T (&UC)[D + 2],
                                               T (&slope)[D][D + 2]) {
    constexpr int NV = D + 2;
    const int bx = sc<D>(0, Lc[0]), by = sc<D>(1, Lc[1]), bz = sc<D>(2, Lc[2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) UC[v] = U[slot_index(g, Q, v, bz, by, bx)];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int ex = d == 0, ey = d == 1, ez = d == 2;
        // C +- e_d outside Q: see NBR_READS
        long long ip = slot_index(g, Q, 0, bz + ez, by + ey, bx + ex);
        long long im = slot_index(g, Q, 0, bz - ez, by - ey, bx - ex);
        if (NBR_READS && Lc[d] == N - 1) {
            const int qn = g.nbr[Q * NBR + 13 + (d == 0 ? 1 : (d == 1 ? 3 : 9))];
            if (qn >= 0) ip = slot_index(g, qn, 0, bz - (N - 1) * ez, by - (N - 1) * ey, bx - (N - 1) * ex);
        }
        if (NBR_READS && Lc[d] == 0) {
            const int qn = g.nbr[Q * NBR + 13 - (d == 0 ? 1 : (d == 1 ? 3 : 9))];
            if (qn >= 0) im = slot_index(g, qn, 0, bz + (N - 1) * ez, by + (N - 1) * ey, bx + (N - 1) * ex);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T up = U[ip + (long long)v * g.slot_elems];
            const T um = U[im + (long long)v * g.slot_elems];
            const T a = up - UC[v];
            const T b = UC[v] - um;
            const T pick = fabs(a) <= fabs(b) ? a : b;
            slope[d][v] = (a * b <= T(0)) ? T(0) : pick;
        }
    }
}

// value of child ch of C: U_C + sum_d (+-1/4) s_d, dims in order
template <typename T, int D>
__device__ __forceinline__ void prolong_child(const T (&UC)[D + 2], const T (&slope)[D][D + 2], int ch,
                                              T (&v)[D + 2]) {
#pragma unroll
    for (int k = 0; k < D + 2; ++k) v[k] = UC[k];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const bool up = (ch >> d) & 1;
#pragma unroll
        for (int k = 0; k < D + 2; ++k) v[k] = up ? v[k] + T(0.25) * slope[d][k] : v[k] - T(0.25) * slope[d][k];
    }
}

// every child of C has rho > 0 and p > 0
template <typename T, int D>
__device__ __forceinline__ bool prolong_positive(const Grid& g, const T (&UC)[D + 2], const T (&slope)[D][D + 2]) {
    const T gm1 = T(g.gamma) - T(1);
    bool ok = true;
#pragma unroll
    for (int ch = 0; ch < (1 << D); ++ch) {
        T v[D + 2];
        prolong_child<T, D>(UC, slope, ch, v);
        T rho, u[D], p, Tt;
        primitives<T, D>(v, gm1, rho, u, p, Tt);
        ok = ok && (rho > T(0)) && (p > T(0));
    }
    return ok;
}

template <typename T, int D, int N, bool NBR_READS>
__device__ void prolong_cell(const Grid& g, const T* U, const PatchMeta& m, const int* l, T* out) {
    constexpr int NV = D + 2;
    int Lc[3], s[3];
    const int Q = prolong_locate<D, N>(m, l, Lc, s);
    if (Q < 0) {
        atomicOr(&g.time->err, ERR_MESH);
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = T(0);
        return;
    }
    T UC[NV], slope[D][NV];
    prolong_slopes<T, D, N, NBR_READS>(g, U, Q, Lc, UC, slope);
    const bool ok = prolong_positive<T, D>(g, UC, slope);
    int mine = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) mine |= s[d] << d;
    T chosen[NV];
    prolong_child<T, D>(UC, slope, mine, chosen);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = ok ? chosen[k] : UC[k];
}

// value of an in-domain cell of a patch: interior, same-level neighbour or prolongation
template <typename T, int D, int N>
__device__ void in_domain_value(const Grid& g, const T* U, const PatchMeta& m, const int* l, T* out) {
    constexpr int NV = D + 2;
    const int slot = m.slot;
    int o[3] = {0, 0, 0};
    bool inside = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        o[d] = l[d] < 0 ? -1 : (l[d] >= N ? 1 : 0);
        inside = inside && o[d] == 0;
    }
    if (inside) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
            out[v] = U[slot_index(g, slot, v, sc<D>(2, l[2]), sc<D>(1, l[1]), sc<D>(0, l[0]))];
        return;
    }
    const int nb = m.nbr[(o[2] + 1) * 9 + (o[1] + 1) * 3 + (o[0] + 1)];
    if (nb >= 0) {
        const int sx = sc<D>(0, l[0] - o[0] * N), sy = sc<D>(1, l[1] - o[1] * N), sz = sc<D>(2, l[2] - o[2] * N);
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = U[slot_index(g, nb, v, sz, sy, sx)];
        return;
    }
    prolong_cell<T, D, N, true>(g, U, m, l, out);
}

// Ghost value of local cell l of a patch: physical boundary rules applied from
// the highest out-of-domain dimension down (the outcome of filling the
// boundary dimension by dimension in the order x, y, z), then the in-domain
// value of the mapped cell.
template <typename T, int D, int N>
__device__ void ghost_value(const Grid& g, const T* U, const PatchMeta& m, int* l, double t, T* out,
                            const double* pre, const double* post) {
    constexpr int NV = D + 2;
    const int lev = m.lev;
    const int* c = m.c;
    int neg = 0;
    for (int it = 0; it < D; ++it) {
        int dd = -1, side = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            if (dd >= 0 || g.periodic[d]) continue;
            const int Gd = c[d] * N + l[d];
            const int n = g.ext[lev][d] * N;
            if (Gd < 0) { dd = d; side = 0; }
            else if (Gd >= n) { dd = d; side = 1; }
        }
        if (dd < 0) break;
        const int kind = g.bc[dd][side];
        const int Gd = c[dd] * N + l[dd];
        const int n = g.ext[lev][dd] * N;
        bool dirichlet = false, behind = false;
        if (kind == AMR_BC_DMR_INFLOW) {
            dirichlet = true;
            behind = true;
        } else if (kind == AMR_BC_DMR_BOTTOM || kind == AMR_BC_DMR_TOP) {
            const double x = g.lo[0] + ((double)(c[0] * N + l[0]) + 0.5) * g.dx[lev][0];
            if (kind == AMR_BC_DMR_BOTTOM) {
                behind = x < 1.0 / 6.0;
                dirichlet = behind;
            } else {
                behind = x < 1.0 / 6.0 + (1.0 + 20.0 * t) / sqrt(3.0);
                dirichlet = true;
            }
        }
        if (dirichlet) {
            const double* st = behind ? post : pre;     // (rho, u, v, p)
            const double r = st[0], ux = st[1], uy = st[2], pp = st[3];
            const double usq = ux * ux + uy * uy;
            double Uc[4];
            Uc[0] = r;
            Uc[1] = r * ux;
            Uc[2] = r * uy;
            Uc[3] = pp / (g.gamma - 1.0) + 0.5 * r * usq;
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v] = T(v < 4 ? Uc[v] : 0.0);
#pragma unroll
            for (int d = 0; d < D; ++d)
                if ((neg >> d) & 1) out[1 + d] = -out[1 + d];
            return;
        }
        int Gs;
        if (kind == AMR_BC_OUTFLOW) {
            Gs = side ? n - 1 : 0;
        } else {                                   // reflecting wall (also DMR bottom beyond 1/6)
            Gs = side ? 2 * n - 1 - Gd : -1 - Gd;
            neg ^= 1 << dd;
        }
        l[dd] = Gs - c[dd] * N;
    }
    in_domain_value<T, D, N>(g, U, m, l, out);
#pragma unroll
    for (int d = 0; d < D; ++d)
        if ((neg >> d) & 1) out[1 + d] = -out[1 + d];
}

// ---------------------------------------------------------------------------
// K1-K3: ghost fill of every patch of one level. The regrid fills every ghost
// cell (the slot-order table); a stage (stage_only) fills the face boxes that
// have no same-level neighbour across them (coarse-fine and domain sides),
// whose cells the RHS reads from the slot (the box-order table that follows
// the first). A work item is a patch and a run of
// `chunk` cells (the size is a launch parameter chosen by the autotuner),
// taken by one warp, which stages the patch's metadata in its own
// shared-memory copy; warps never wait for one another.
// ---------------------------------------------------------------------------
template <typename T, int D, int N, bool STAGE>
__global__ void __launch_bounds__(256, STAGE && sizeof(T) == 4 ? 3 : 0) k_ghost(Grid g, T* U, int level, double tfrac, int one_slot,
                                               double4 pre, double4 post, int chunk, int n_cells) {
    constexpr bool stage_only = STAGE;                  // compiled apart: the full fill keeps its registers
    constexpr int NV = D + 2;
    __shared__ PatchMeta metas[256 / 32];
    if (g.time->cancel) return;                          // a void step (see DevTime::cancel)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    PatchMeta& m = metas[warp];
    const int lo = g.level_off[level], hi = g.level_off[level + 1];
    const int npatch = one_slot >= 0 ? 1 : hi - lo;
    const double t = g.time->t + tfrac * g.time->dt;
    const double pr[4] = {pre.x, pre.y, pre.z, pre.w};
    const double po[4] = {post.x, post.y, post.z, post.w};
    // a stage walks the 2d face boxes of a patch (G N^(d-1) table entries
    // each) and skips a box whole when a same-level neighbour lies across it
    constexpr int BOX = G * (D == 1 ? 1 : (D == 2 ? N : N * N));
    const int* tab = stage_only ? g.ghost_tab + g.n_ghost : g.ghost_tab;   // box order, or slot order
    const int span = stage_only ? BOX : n_cells;          // table entries one run of items covers
    const int nruns = stage_only ? 2 * D : 1;
    const int nchunk = (span + chunk - 1) / chunk;        // chunk: ghost cells per work item
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int item = blockIdx.x * (blockDim.x >> 5) + warp; item < npatch * nruns * nchunk; item += nw) {
        const int pi = item / (nruns * nchunk);
        const int rest = item - pi * nruns * nchunk;
        const int run = rest / nchunk;
        const int g0 = run * span + (rest - run * nchunk) * chunk;
        const int g1 = min(g0 + chunk, run * span + span);
        const int slot = one_slot >= 0 ? one_slot : g.all_list[lo + pi];
        if (stage_only) {
            const int d = run >> 1, side = run & 1;
            const int across = g.nbr[slot * NBR + 13 + (side ? 1 : -1) * (d == 0 ? 1 : (d == 1 ? 3 : 9))];
            if (across >= 0) continue;
            if constexpr (STAGE) if (across == -1) {
                // in the domain without a same-level patch: every cell of the box
                // is prolonged; per coarse cell C of the box (2 layers along d,
                // H^(d-1) across) one slope evaluation and positivity test, then
                // the 4 or 8 children of C in the box are written, each with the
                // value the per-cell path gives it
                constexpr int H = N / 2;
                constexpr int HT = D == 1 ? 1 : (D == 2 ? H : H * H);
                constexpr int NCB = 2 * HT;
                const int per = (NCB + nchunk - 1) / nchunk;
                const int q0 = (rest - run * nchunk) * per, q1 = min(q0 + per, NCB);
                load_meta_warp(g, slot, m);
                for (int qc = q0 + lane; qc < q1; qc += 32) {
                    const int layer = qc / HT, tq = qc - layer * HT;
                    // a fine cell of the box among C's children (local coordinates)
                    int l[3] = {0, 0, 0};
                    const int t1 = tq % H, t2 = tq / H;
                    int ti = 0;
#pragma unroll
                    for (int e = 0; e < D; ++e) {
                        if (e == d) l[e] = side ? (layer ? N + 2 : N) : (layer ? -3 : -1);
                        else l[e] = 2 * (ti++ == 0 ? t1 : t2);
                    }
                    int Lc[3], sr[3];
                    const int Q = prolong_locate<D, N>(m, l, Lc, sr);
                    T UC[NV], slope[D][NV];
                    bool ok = false;
                    if (Q < 0) {
                        atomicOr(&g.time->err, ERR_MESH);
                    } else {
                        prolong_slopes<T, D, N, true>(g, U, Q, Lc, UC, slope);
                        ok = prolong_positive<T, D>(g, UC, slope);
                    }
#pragma unroll
                    for (int ch = 0; ch < (1 << D); ++ch) {
                        int lc[3] = {0, 0, 0};
                        bool in = true;
#pragma unroll
                        for (int e = 0; e < D; ++e) {
                            lc[e] = l[e] - sr[e] + ((ch >> e) & 1);
                            in = in && (e == d ? (side ? lc[e] >= N && lc[e] < N + G : lc[e] >= -G && lc[e] < 0)
                                               : lc[e] >= 0 && lc[e] < N);
                        }
                        if (!in) continue;
                        T val[NV];
                        if (Q < 0) {
#pragma unroll
                            for (int v = 0; v < NV; ++v) val[v] = T(0);
                        } else if (ok) {
                            prolong_child<T, D>(UC, slope, ch, val);
                        } else {
#pragma unroll
                            for (int v = 0; v < NV; ++v) val[v] = UC[v];
                        }
#pragma unroll
                        for (int v = 0; v < NV; ++v)
                            U[slot_index(g, slot, v, sc<D>(2, lc[2]), sc<D>(1, lc[1]), sc<D>(0, lc[0]))] = val[v];
                    }
                }
                __syncwarp();                            // the copy is read until here
                continue;
            }
        }
        load_meta_warp(g, slot, m);
        for (int gi = g0 + lane; gi < g1; gi += 32) {
            const int pk = tab[gi];
            int l[3] = {(pk & 1023) - G, ((pk >> 10) & 1023) - G, ((pk >> 20) & 1023) - G};
            const int sx = l[0] + G, sy = D >= 2 ? l[1] + G : 0, sz = D == 3 ? l[2] + G : 0;
            T val[NV];
            ghost_value<T, D, N>(g, U, m, l, t, val, pr, po);
#pragma unroll
            for (int v = 0; v < NV; ++v) U[slot_index(g, slot, v, sz, sy, sx)] = val[v];
        }
        __syncwarp();                                    // the copy is read until here
    }
}

// Restriction mean of the 2^d children of a covered coarse cell, given in
// lexicographic z, y, x order: (sum) * 2^-d, summed in FP64 (FP32 fields: an
// error-free FP32 pair sum, rounded once). Shared by the restriction kernel
// and the fused restriction of the RHS, so both give the same bits.
template <typename T, int D>
__device__ __forceinline__ T restrict_mean(const T (&ch)[1 << D]) {
    constexpr int NCH = 1 << D;
    constexpr double scale = D == 1 ? 0.5 : (D == 2 ? 0.25 : 0.125);
    if constexpr (sizeof(T) == 4) {
        // FP32 fields: the sum carried as an unevaluated pair s + e (Knuth's
        // TwoSum adds each child without error into s and collects the
        // rounding errors in e), rounded once; equal to the FP64 sum rounded
        // to FP32 up to near-ties, at FP32 cost
        float sum = ch[0], err = 0.0f;
#pragma unroll
        for (int k = 1; k < NCH; ++k) {
            const float a = ch[k];
            const float t = __fadd_rn(sum, a);
            const float bv = __fsub_rn(t, sum);
            const float e = __fadd_rn(__fsub_rn(sum, __fsub_rn(t, bv)), __fsub_rn(a, bv));
            sum = t;
            err = __fadd_rn(err, e);
        }
        return __fmul_rn(__fadd_rn(sum, err), (float)scale);
    } else {
        double acc = (double)ch[0];
#pragma unroll
        for (int k = 1; k < NCH; ++k) acc = acc + (double)ch[k];
        return T(acc * scale);
    }
}

// ---------------------------------------------------------------------------
// K4: fused right-hand side and SSP-RK3 stage of a chunk of one leaf patch.
// The chunk (DZ planes in 3D, the whole patch in 1D/2D) plus its ghost halo
// is staged in shared memory as primitives (p, u_0.., T); face fluxes of one
// dimension at a time go to a shared buffer; each thread accumulates the
// divergence of its own cells in registers, then writes
// U_out = a U0 + b (U_s + dt R)  (a = 0, b = 1 in stage 1).
// fuse_restrict: a chunk of a patch of the finest level L - 1 (>= 1) also
// restricts its updated cells into the parent (restrict_mean, as the
// restriction kernel does): the finest level is never the coarse side of a
// reflux, so its stage output is final here, and its parent, whose cells are
// all covered, is neither read by this launch nor refluxed.
// ---------------------------------------------------------------------------
// EXT: extra faces per dimension beyond the N + 1 of a patch row (2 for the
// central scheme, whose divergence reads the faces at i -+ 3/2)
// PADQ: per-variable blocks and the halo block start on 128-byte boundaries
// (the halo planes are then tensor-copy destinations)
template <int D, int N, int DZ, int EXT = 0, bool PADQ = false> struct Chunk {
    static constexpr int S = N + 2 * G;
    static constexpr int CX = N, CY = D >= 2 ? N : 1, CZ = D == 3 ? DZ : 1;
    // staged cells per variable: 1D/2D the whole slot; 3D the DZ centre planes
    // in full (S x S) and the 2G halo planes only over the interior N x N, the
    // only part the z-faces read
    static constexpr int QX = S, QY = D >= 2 ? S : 1, QZ = D == 3 ? DZ : 1;
    static constexpr int QC = PADQ ? (QX * QY * QZ + 31) / 32 * 32 : QX * QY * QZ;   // centre cells
    static constexpr int QH = D == 3 ? 2 * G * N * N : 0;         // compact halo cells
    static constexpr int QN = PADQ ? (QC + QH + 31) / 32 * 32 : QC + QH;
    static constexpr int CELLS = CX * CY * CZ;
    static constexpr int NCH = D == 3 ? N / DZ : 1;
    static constexpr int F0 = (CX + 1 + EXT) * CY * CZ;
    static constexpr int F1 = D >= 2 ? CX * (CY + 1 + EXT) * CZ : 0;
    static constexpr int F2 = D == 3 ? CX * CY * (CZ + 1 + EXT) : 0;
    // face buffer: the x and y faces of a chunk together, then the z faces
    static constexpr int FMAX = F0 + F1 > F2 ? F0 + F1 : F2;
    // face rows per dimension d (x extent FX_d, y extent FY_d) and their
    // multiply-high reciprocals
    static constexpr int FX0 = CX + 1 + EXT, FX1 = CX, FX2 = CX;
    static constexpr int FY0 = CY, FY1 = CY + 1 + EXT, FY2 = CY;
    static constexpr unsigned MX0 = 0xFFFFFFFFu / FX0 + 1u, MX1 = 0xFFFFFFFFu / FX1 + 1u, MX2 = MX1;
    static constexpr unsigned MY0 = 0xFFFFFFFFu / FY0 + 1u, MY1 = 0xFFFFFFFFu / FY1 + 1u, MY2 = MY0;
    static constexpr int TRANS = D == 1 ? 1 : (D == 2 ? N : N * N);   // cells on a patch face
};

template <typename T, int D, int N, int DZ, int FLUX, bool TMA = false>
constexpr size_t rhs_smem_bytes() {
    using C = Chunk<D, N, DZ, FLUX == AMR_FLUX_CENTRAL ? 2 : 0, TMA>;
    // TMA: 128 bytes to align the base, an mbarrier and an abort word
    return sizeof(T) * ((size_t)(D + 2) * C::QN + (size_t)(D + 2) * C::FMAX) + (TMA ? 128 + 16 : 0);
}

// Tensor copies (TMA) of the halo planes: a 4D tiled load of a box into
// shared memory, completing on an mbarrier with a transaction count
__device__ __forceinline__ uint32_t rhs_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void rhs_tma_load4(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                              uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void rhs_mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar), "r"(bytes)
                 : "memory");
}
// wait for phase `parity` of the mbarrier: false once *abort is set, or after
// TC_WAIT_CYCLES SM cycles (which sets *abort), so a copy that never lands
// costs one bounded wait per CTA, not one per work item
__device__ __forceinline__ bool rhs_mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
        if ((it & 63u) == 63u && clock64() - t0 > TC_WAIT_CYCLES) {
            *abort = 1;
            return false;
        }
    }
}

// TMA (3D, DZ >= 4): the 2G halo planes of a chunk arrive by tensor copies,
// one 16 x 16 x 3 box per variable and side (each box has one source slot:
// the same-level neighbour across z or the slot itself), issued by thread 0
// while the other threads stage the centre planes; they land as conserved
// variables in the halo block and are converted to primitives in place.
template <typename T, int D, int N, int DZ, int NTH, int MINB, int FLUX, bool TMA = false>
__global__ void __launch_bounds__(NTH, MINB) k_rhs(Grid g, const T* __restrict__ Us, const T* U0,
                                             T* Uout, T* __restrict__ faces,
                                             int stage, int one_slot, int fuse_restrict,
                                             const __grid_constant__ CUtensorMap tmap) {
    constexpr bool CEN = FLUX == AMR_FLUX_CENTRAL;
    constexpr int EXT = CEN ? 2 : 0;                   // central: faces i - 3/2 .. N + 1/2 along d
    static_assert(!TMA || (D == 3 && DZ >= 4 && sizeof(T) == 4 && !CEN), "halo boxes with one source slot");
    using C = Chunk<D, N, DZ, EXT, TMA>;
    constexpr int NV = D + 2;
    constexpr int NT = D - 1;
    constexpr int CPT = (C::CELLS + NTH - 1) / NTH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (g.time->cancel) return;                          // a void step (see DevTime::cancel)
    unsigned char* sbase = smem_raw;
    if constexpr (TMA)                                   // tensor-copy destinations: 128-byte aligned
        sbase += (128u - (rhs_smem_addr(smem_raw) & 127u)) & 127u;
    T* q = reinterpret_cast<T*>(sbase);                    // [NV][QZ][QY][QX]
    T* Fs = q + NV * C::QN;                               // [NV][FMAX]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Fs + NV * C::FMAX);   // TMA: the halo copies' barrier
    volatile int* tabort = reinterpret_cast<volatile int*>(mbar + 1);  // TMA: a wait gave up
    uint32_t tparity = 0;
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(rhs_smem_addr(mbar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            *tabort = 0;
        }
        __syncthreads();
    }
    const T gamma = T(g.gamma);
    const T gm1 = T(g.gamma) - T(1);
    const double dtd = g.time->dt;
    const T dt = T(dtd);
    const T ra = stage == 0 ? T(0) : (stage == 1 ? T(0.75) : T(1.0 / 3.0));
    const T rb = stage == 0 ? T(1) : (stage == 1 ? T(0.25) : T(2.0 / 3.0));
    // leaves only: a patch with children is covered by them, and the
    // restriction after the stage overwrites its whole interior
    const int npatch = one_slot >= 0 ? 1 : g.counts[1];
    const int n_items = npatch * C::NCH;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int pi = item / C::NCH;
        const int z0 = (item - pi * C::NCH) * DZ;        // first interior plane of the chunk (3D)
        const int slot = one_slot >= 0 ? one_slot : g.leaf_list[pi];
        const int lev = g.level[slot];
        const int pf = g.pflag[slot];
        const bool fuse = fuse_restrict && lev == g.L - 1 && lev >= 1;
        // 1. stage the chunk and its halo as primitives, loading 16-byte vectors
        //    along x (slot rows are 16-byte aligned)
        {
            constexpr int VE = 16 / sizeof(T);
            auto stage = [&](const T (&Uv)[NV][VE], int e, int qidx) {
                T Uc[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) Uc[v] = Uv[v][e];
                T rho, u[D], p, Tt;
                primitives<T, D>(Uc, gm1, rho, u, p, Tt);
                q[qidx] = p;
#pragma unroll
                for (int d = 0; d < D; ++d) q[(1 + d) * C::QN + qidx] = u[d];
                q[(D + 1) * C::QN + qidx] = Tt;
            };
            auto loadv = [&](T (&Uv)[NV][VE], int src, int sz, int sy, int sx) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const T* p = Us + slot_index(g, src, v, sz, sy, sx);
                    if constexpr (sizeof(T) == 4) {
                        const float4 t4 = *reinterpret_cast<const float4*>(p);
                        Uv[v][0] = t4.x; Uv[v][1] = t4.y; Uv[v][2] = t4.z; Uv[v][3] = t4.w;
                    } else {
                        const double2 t2 = *reinterpret_cast<const double2*>(p);
                        Uv[v][0] = t2.x; Uv[v][1] = t2.y;
                    }
                }
            };
            // face ghosts come from the same-level neighbour across the face
            // when it exists (the stage's ghost fill leaves them unfilled),
            // else from the slot's own ghost cells: neighbour slot and the
            // shift of the slot coordinate along that dimension
            auto across = [&](int d, int side, int& src, int& shift) {
                const int nb = g.nbr[slot * NBR + 13 + (side ? 1 : -1) * (d == 0 ? 1 : (d == 1 ? 3 : 9))];
                src = nb >= 0 ? nb : slot;
                shift = nb >= 0 ? (side ? -N : N) : 0;
            };
            int sxm, dxm, sxp, dxp, sym = slot, dym = 0, syp = slot, dyp = 0;
            across(0, 0, sxm, dxm);
            across(0, 1, sxp, dxp);
            if constexpr (D >= 2) {
                across(1, 0, sym, dym);
                across(1, 1, syp, dyp);
            }
            if constexpr (TMA) {
                // the halo boxes: planes z0 .. z0 + 2 and z0 + DZ + 3 .. + 5 of the
                // slot, from the z neighbour at the patch's ends (DZ >= 4: a box
                // never straddles the interior's edge); interior x and y; the
                // previous item's z faces, the last readers of this block, ended
                // at a barrier this thread has passed
                if (threadIdx.x == 0 && !*tabort) {
                    int szm, dzm, szp, dzp;
                    across(2, 0, szm, dzm);
                    across(2, 1, szp, dzp);
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    const uint32_t mb = rhs_smem_addr(mbar);
                    rhs_mbar_expect(mb, (uint32_t)(NV * C::QH * sizeof(T)));
                    const int zl = z0 == 0 ? z0 + dzm : z0, wl = z0 == 0 ? szm : slot;
                    const int zh = z0 + DZ + G + (z0 + DZ == N ? dzp : 0), wh = z0 + DZ == N ? szp : slot;
                    constexpr int XP = PatchShape<T, N>::XP;
#pragma unroll 1
                    for (int v = 0; v < NV; ++v) {
                        rhs_tma_load4(rhs_smem_addr(q + v * C::QN + C::QC), &tmap, XP + G, G, zl, wl * NV + v, mb);
                        rhs_tma_load4(rhs_smem_addr(q + v * C::QN + C::QC + G * N * N), &tmap, XP + G, G, zh,
                                      wh * NV + v, mb);
                    }
                }
            }
            // centre planes (3D) or the whole slot (1D/2D): full rows; a row
            // outside the interior along y comes whole from its y source (its
            // x ghosts are edge cells, which no face reads)
            // aligned vectors of the padded row covering slot x in [0, QX):
            // vector xv starts at slot x xv VE - XP (negative: the row pad)
            constexpr int XP = PatchShape<T, N>::XP;
            constexpr int XV0 = XP / VE, NXV = (XP + C::QX + VE - 1) / VE - XV0;
#pragma unroll 2
            for (int iv = threadIdx.x; iv < NXV * C::QY * C::QZ; iv += NTH) {
                const int xv = iv % NXV, qy = (iv / NXV) % C::QY, qz = iv / (NXV * C::QY);
                const int sz = D == 3 ? z0 + G + qz : 0;
                const int x0 = (xv + XV0) * VE - XP;
                T Uv[NV][VE];
                const int ly = qy - G;
                if (D >= 2 && (ly < 0 || ly >= N)) {
                    loadv(Uv, ly < 0 ? sym : syp, sz, qy + (ly < 0 ? dym : dyp), x0);
                } else {
                    loadv(Uv, slot, sz, qy, x0);
                    if (x0 < G) {                            // x ghosts below the interior
                        T Wv[NV][VE];
                        loadv(Wv, sxm, sz, qy, x0 + dxm);
#pragma unroll
                        for (int e = 0; e < VE; ++e)
                            if (x0 + e < G) {
#pragma unroll
                                for (int v = 0; v < NV; ++v) Uv[v][e] = Wv[v][e];
                            }
                    }
                    if (x0 + VE > G + N) {                   // x ghosts above the interior
                        T Wv[NV][VE];
                        loadv(Wv, sxp, sz, qy, x0 + dxp);
#pragma unroll
                        for (int e = 0; e < VE; ++e)
                            if (x0 + e >= G + N) {
#pragma unroll
                                for (int v = 0; v < NV; ++v) Uv[v][e] = Wv[v][e];
                            }
                    }
                }
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    const int qx = x0 + e;
                    if (qx >= 0 && qx < C::QX) stage(Uv, e, (qz * C::QY + qy) * C::QX + qx);
                }
            }
            if constexpr (TMA) {
                // the halo boxes have landed: conserved variables -> primitives
                const bool landed = rhs_mbar_wait(rhs_smem_addr(mbar), tparity, tabort);
                tparity ^= 1u;
                if (!landed && threadIdx.x == 0) atomicOr(&g.time->err, ERR_TIMEOUT);
#pragma unroll 2
                for (int c = threadIdx.x; c < C::QH; c += NTH) {
                    const int qidx = C::QC + c;
                    T Uc[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) Uc[v] = q[v * C::QN + qidx];
                    T rho, u[D], p, Tt;
                    primitives<T, D>(Uc, gm1, rho, u, p, Tt);
                    q[qidx] = p;
#pragma unroll
                    for (int d = 0; d < D; ++d) q[(1 + d) * C::QN + qidx] = u[d];
                    q[(D + 1) * C::QN + qidx] = Tt;
                }
                // these generic writes before the next item's tensor copies into
                // the block (ordered by the barriers between)
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            } else if constexpr (D == 3) {
                // halo planes: interior x in [G, G + N), which starts on a
                // 32-byte boundary, as N / VE aligned vectors, from the z
                // source when the plane lies outside the interior
                constexpr int HX0 = G;
                constexpr int NHV = N / VE;
                static_assert(N % VE == 0, "interior rows are whole vectors");
                int szm, dzm, szp, dzp;
                across(2, 0, szm, dzm);
                across(2, 1, szp, dzp);
#pragma unroll 2
                for (int iv = threadIdx.x; iv < NHV * N * 2 * G; iv += NTH) {
                    const int xv = iv % NHV, hy = (iv / NHV) % N, zh = iv / (NHV * N);
                    const int sz = z0 + (zh < G ? zh : zh + DZ);
                    const int lz = sz - G;
                    const int src = lz < 0 ? szm : (lz >= N ? szp : slot);
                    const int shz = lz < 0 ? dzm : (lz >= N ? dzp : 0);
                    T Uv[NV][VE];
                    loadv(Uv, src, sz + shz, hy + G, HX0 + xv * VE);
#pragma unroll
                    for (int e = 0; e < VE; ++e) {
                        const int x = HX0 + xv * VE + e;
                        if (x >= G && x < G + N) stage(Uv, e, C::QC + (zh * N + hy) * N + (x - G));
                    }
                }
            }
        }
        __syncthreads();
        // stages 2-3 read U0 in the update: its interior rows of this chunk
        // into L2 now (last written a step ago, so not in L2), while the
        // face passes run
        if (stage > 0) {
            constexpr int ROWS = NV * C::CZ * C::CY;
            for (int r = threadIdx.x; r < ROWS; r += NTH) {
                const int v = r / (C::CZ * C::CY), rz = (r / C::CY) % C::CZ, ry = r % C::CY;
                const T* a = U0 + slot_index(g, slot, v, D == 3 ? z0 + G + rz : 0, D >= 2 ? ry + G : 0, G);
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a));
            }
        }
        T R[CPT][NV];
        // two phases: the x and y faces of the chunk in one pass (an even
        // share of faces per thread), then the z faces; each phase ends with
        // the divergence of its dimensions, x before y before z. One rolled
        // loop: a single copy of the face-flux code keeps the kernel inside
        // the instruction cache
        constexpr int NPH = D == 3 ? 2 : 1;
#pragma unroll 1
        for (int ph = 0; ph < NPH; ++ph) {
            const int nfp = ph == 0 ? (D >= 2 ? C::F0 + C::F1 : C::F0) : C::F2;
            for (int fp = threadIdx.x; fp < nfp; fp += NTH) {
                // the face's dimension (uniform across a warp except at the one
                // x/y boundary of the buffer when F0 is not a multiple of 32).
                // Node loads and face stores are compiled per dimension, so
                // their shared-memory offsets are constants; the flux code
                // between them exists once
                const int d = ph == 1 ? 2 : (D >= 2 && fp >= C::F0 ? 1 : 0);
                T pp[6], un[6], ut[NT > 0 ? NT : 1][6], Tt[6];
                int fi, fj, fk;
                auto load = [&](auto dc) {
                    constexpr int DD = decltype(dc)::value;
                    constexpr int fbase = DD == 1 ? C::F0 : 0;   // the dimension's faces in the buffer
                    constexpr int FX = DD == 0 ? C::FX0 : (DD == 1 ? C::FX1 : C::FX2);
                    constexpr int FY = DD == 0 ? C::FY0 : (DD == 1 ? C::FY1 : C::FY2);
                    // f -> (fi, fj, fk) by multiply-high division, exact for f * FX < 2^32
                    constexpr unsigned mFX = DD == 0 ? C::MX0 : (DD == 1 ? C::MX1 : C::MX2);
                    constexpr unsigned mFY = DD == 0 ? C::MY0 : (DD == 1 ? C::MY1 : C::MY2);
                    constexpr int step = DD == 0 ? 1 : C::QX;     // x and y pencils stay in one centre plane
                    // tangential velocity components in increasing dimension order
                    [[maybe_unused]] constexpr int t1 = DD == 0 ? 1 : 0;
                    [[maybe_unused]] constexpr int t2 = DD == 2 ? 1 : 2;
                    const int f = fp - fbase;
                    const int q1 = (int)__umulhi((unsigned)f, mFX);
                    fk = D == 1 ? 0 : (int)__umulhi((unsigned)q1, mFY);   // 1D: FY = FZ = 1
                    fi = f - q1 * FX;
                    fj = q1 - fk * FY;
                    // smem index of pencil node 0 (cell index - 3 along d; G = 3).
                    // Central: face index a along d is the face i - 1/2 of cell
                    // i = a - 1, and only nodes 1..4 (cells i - 2 .. i + 1) are read
                    int base = 0;
                    if constexpr (DD < 2) {
                        const int bx = fi + G - (DD == 0 ? G + EXT / 2 : 0);
                        const int by = (D >= 2 ? fj + G : 0) - (DD == 1 ? G + EXT / 2 : 0);
                        base = ((D == 3 ? fk : 0) * C::QY + by) * C::QX + bx;
                    }
#pragma unroll
                    for (int k = CEN ? 1 : 0; k < (CEN ? 5 : 6); ++k) {
                        int id;
                        if constexpr (DD < 2) {
                            id = base + k * step;
                        } else {                                 // z pencil: halo plane or centre plane
                            const int zz = fk + k - EXT / 2;     // staged z index 0 .. DZ + 5
                            id = (zz >= G && zz < G + DZ)
                                     ? ((zz - G) * C::QY + fj + G) * C::QX + fi + G
                                     : C::QC + ((zz < G ? zz : zz - DZ) * N + fj) * N + fi;
                        }
                        pp[k] = q[id];
                        un[k] = q[(1 + DD) * C::QN + id];
                        Tt[k] = q[(D + 1) * C::QN + id];
                        if constexpr (NT >= 1) ut[0][k] = q[(1 + t1) * C::QN + id];
                        if constexpr (NT >= 2) ut[NT > 1 ? 1 : 0][k] = q[(1 + t2) * C::QN + id];
                    }
                };
                if constexpr (D == 3) {
                    if (d == 2) load(std::integral_constant<int, 2>{});
                    else if (d == 1) load(std::integral_constant<int, 1>{});
                    else load(std::integral_constant<int, 0>{});
                } else if constexpr (D == 2) {
                    if (d == 1) load(std::integral_constant<int, 1>{});
                    else load(std::integral_constant<int, 0>{});
                } else {
                    load(std::integral_constant<int, 0>{});
                }
                T Fp[NT + 3];
                if constexpr (CEN) central_flux<T, NT>(pp, un, ut, Tt, gm1, Fp);
                else if constexpr (FLUX == AMR_FLUX_HYBRID) hybrid_flux<T, NT>(pp, un, ut, Tt, gamma, gm1, T(g.theta_sw), Fp);
                else if constexpr (sizeof(T) == 4 && FLUX == AMR_FLUX_RUSANOV)
                    face_flux_x2<NT>(pp, un, ut, Tt, gamma, gm1, Fp);
                else face_flux<T, NT, FLUX>(pp, un, ut, Tt, gamma, gm1, Fp);
                auto store = [&](auto dc) {
                    constexpr int DD = decltype(dc)::value;
                    constexpr int t1 = DD == 0 ? 1 : 0;
                    // pencil order -> global variable order
                    T Fg[NV];
                    Fg[0] = Fp[0];
#pragma unroll
                    for (int e = 0; e < D; ++e)
                        Fg[1 + e] = e == DD ? Fp[1] : (e == t1 ? Fp[NT >= 1 ? 2 : 1] : Fp[NT >= 2 ? 3 : 1]);
                    Fg[NV - 1] = Fp[NT + 2];
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fs[v * C::FMAX + fp] = Fg[v];
                    // patch-boundary faces needed by the coarse-fine flux correction
                    // (central: the conservative face values, saved by the divergence)
                    const int fd = DD == 0 ? fi : (DD == 1 ? fj : fk + z0);
                    const int side = fd == 0 ? 0 : (fd == N ? 1 : -1);
                    if (!CEN && side >= 0 && ((pf >> (8 + 2 * DD + side)) & 1)) {
                        int tidx;
                        if constexpr (D == 1) tidx = 0;
                        else if constexpr (D == 2) tidx = DD == 0 ? fj : fi;
                        else tidx = DD == 0 ? (fk + z0) * N + fj : (DD == 1 ? (fk + z0) * N + fi : fj * N + fi);
                        T* dst = faces + ((long long)slot * 2 * D + 2 * DD + side) * NV * C::TRANS + tidx;
#pragma unroll
                        for (int v = 0; v < NV; ++v) dst[v * C::TRANS] = Fg[v];
                    }
                };
                if constexpr (D == 3) {
                    if (d == 2) store(std::integral_constant<int, 2>{});
                    else if (d == 1) store(std::integral_constant<int, 1>{});
                    else store(std::integral_constant<int, 0>{});
                } else if constexpr (D == 2) {
                    if (d == 1) store(std::integral_constant<int, 1>{});
                    else store(std::integral_constant<int, 0>{});
                } else {
                    store(std::integral_constant<int, 0>{});
                }
            }
            __syncthreads();
            // divergence of the phase's dimensions, each compiled for its own
            // dimension (constant face strides)
            auto divergence = [&](auto dc) {
                constexpr int d = decltype(dc)::value;
                constexpr int FX = d == 0 ? C::FX0 : (d == 1 ? C::FX1 : C::FX2);
                constexpr int FY = d == 0 ? C::FY0 : (d == 1 ? C::FY1 : C::FY2);
                const T* Fd = Fs + (d == 1 ? C::F0 : 0);
                const T dxd = T(g.dx[lev][d]);
                const T idx = T(1) / dxd;                        // FP32: multiply by the reciprocal
                constexpr int fstep = d == 0 ? 1 : (d == 1 ? FX : FX * FY);
#pragma unroll
                for (int n = 0; n < CPT; ++n) {
                    const int cidx = threadIdx.x + n * NTH;
                    if (cidx < C::CELLS) {
                        const int ci = cidx % C::CX;
                        const int cj = (cidx / C::CX) % C::CY;
                        const int ck = cidx / (C::CX * C::CY);
                        const int flo = (ck * FY + cj) * FX + ci + (CEN ? fstep : 0);
                        const int fhi = flo + fstep;
                        if constexpr (CEN) {
                            // Eq. 9 as the difference of G = (26 F_f - F_{f-1} - F_{f+1}) / 24
                            const int cd = d == 0 ? ci : (d == 1 ? cj : ck + z0);
                            const int side = cd == 0 ? 0 : (cd == N - 1 ? 1 : -1);
                            const bool save = side >= 0 && ((pf >> (8 + 2 * d + side)) & 1);
                            T* dst = nullptr;
                            if (save) {
                                int tidx;
                                if (D == 1) tidx = 0;
                                else if (D == 2) tidx = d == 0 ? cj : ci;
                                else tidx = d == 0 ? (ck + z0) * N + cj : (d == 1 ? (ck + z0) * N + ci : cj * N + ci);
                                dst = faces + ((long long)slot * 2 * D + 2 * d + side) * NV * C::TRANS + tidx;
                            }
#pragma unroll
                            for (int v = 0; v < NV; ++v) {
                                const T* Fv = Fd + v * C::FMAX;
                                const T flo_m = Fv[flo - fstep], flo_c = Fv[flo], fhi_c = Fv[fhi], fhi_p = Fv[fhi + fstep];
                                T glo = T(26) * flo_c - flo_m - fhi_c;
                                T ghi = T(26) * fhi_c - flo_c - fhi_p;
                                if constexpr (sizeof(T) == 4) { glo = glo * T(1.0 / 24.0); ghi = ghi * T(1.0 / 24.0); }
                                else { glo = glo / T(24); ghi = ghi / T(24); }
                                if (save) dst[v * C::TRANS] = side ? ghi : glo;
                                const T df = ghi - glo;
                                const T dv = sizeof(T) == 4 ? df * idx : df / dxd;
                                R[n][v] = d == 0 ? -dv : R[n][v] - dv;
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < NV; ++v) {
                                const T df = Fd[v * C::FMAX + fhi] - Fd[v * C::FMAX + flo];
                                const T dv = sizeof(T) == 4 ? df * idx : df / dxd;
                                R[n][v] = d == 0 ? -dv : R[n][v] - dv;
                            }
                        }
                    }
                }
            };
            if (ph == 0) {
                divergence(std::integral_constant<int, 0>{});
                if constexpr (D >= 2) divergence(std::integral_constant<int, 1>{});
            } else if constexpr (D == 3) {
                divergence(std::integral_constant<int, 2>{});
            }
            // the next phase's faces overwrite the face buffer, and so does a
            // fused restriction's copy of the update; otherwise no barrier is
            // needed after the last phase: the update touches no shared
            // memory, the next item's staging writes only the primitives
            // (which no divergence reads), and its face pass starts after the
            // barrier that ends that staging, which every thread reaches only
            // after its divergence here
            if (ph + 1 < NPH || fuse) __syncthreads();
        }
        // 3. stage update of the chunk's cells
#pragma unroll
        for (int n = 0; n < CPT; ++n) {
            const int cidx = threadIdx.x + n * NTH;
            if (cidx < C::CELLS) {
                const int ci = cidx % C::CX;
                const int cj = (cidx / C::CX) % C::CY;
                const int ck = cidx / (C::CX * C::CY);
                const int sx = ci + G, sy = D >= 2 ? cj + G : 0, sz = D == 3 ? z0 + ck + G : 0;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const long long id = slot_index(g, slot, v, sz, sy, sx);
                    const T us = Us[id];
                    T o;
                    if (stage == 0) o = us + dt * R[n][v];
                    else o = ra * U0[id] + rb * (us + dt * R[n][v]);
                    Uout[id] = o;
                    if (fuse) Fs[v * C::CELLS + cidx] = o;   // the chunk's output, [v][z][y][x]
                }
            }
        }
        // 4. fused restriction of the chunk's cells into the parent
        if (fuse) {
            constexpr int H = N / 2;
            constexpr int HZ = D == 3 ? DZ / 2 : 1, HY = D >= 2 ? H : 1;
            constexpr int NCC = HZ * HY * H;                // coarse cells of the chunk
            static_assert(D < 3 || DZ % 2 == 0, "chunks hold whole coarse planes");
            __syncthreads();
            const int par = g.parent[slot];
            if (par < 0) {
                if (threadIdx.x == 0) atomicOr(&g.time->err, ERR_MESH);
            } else {
                const int ox = (g.coord[slot * 3 + 0] & 1) * H;
                const int oy = D >= 2 ? (g.coord[slot * 3 + 1] & 1) * H : 0;
                const int oz = D == 3 ? (g.coord[slot * 3 + 2] & 1) * H + z0 / 2 : 0;
                for (int c = threadIdx.x; c < NV * NCC; c += NTH) {
                    const int v = c / NCC, r = c - v * NCC;
                    const int cx = r % H, cy = (r / H) % HY, cz = r / (H * HY);
                    T ch[1 << D];                           // children in lexicographic z, y, x order
#pragma unroll
                    for (int k = 0; k < (1 << D); ++k) {
                        const int ax = k & 1, ay = D >= 2 ? (k >> 1) & 1 : 0, az = D == 3 ? k >> 2 : 0;
                        ch[k] = Fs[v * C::CELLS + ((2 * cz + az) * C::CY + 2 * cy + ay) * C::CX + 2 * cx + ax];
                    }
                    Uout[slot_index(g, par, v, D == 3 ? oz + cz + G : 0, D >= 2 ? oy + cy + G : 0, ox + cx + G)] =
                        restrict_mean<T, D>(ch);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K5: coarse-fine flux correction. For each leaf patch with a face whose
// same-level neighbour has children, the coarse face flux F_c is replaced by
// the mean F_f of the 2^(d-1) fine face fluxes (summed in lexicographic
// z, y, x order, times 2^-(d-1)), applied to the stage result as
// U -/+ b dt (F_f - F_c) / dx on the high/low face; faces x-, x+, y-, ... in turn.
// ---------------------------------------------------------------------------
template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_reflux(Grid g, T* Uout, const T* __restrict__ faces, int stage,
                                                int one_item) {
    constexpr int NV = D + 2;
    constexpr int TRANS = Chunk<D, N, 1>::TRANS;
    if (g.time->cancel) return;                          // a void step (see DevTime::cancel)
    const T rb = stage == 0 ? T(1) : (stage == 1 ? T(0.25) : T(2.0 / 3.0));
    const T dt = T(g.time->dt);
    const int n = one_item >= 0 ? one_item + 1 : g.counts[2];
    for (int e = one_item >= 0 ? one_item : blockIdx.x; e < n; e += gridDim.x) {
        const int slot = g.reflux_list[e];
        const int lev = g.level[slot];
        for (int d = 0; d < D; ++d) {
            for (int side = 0; side < 2; ++side) {
                const int* fs = g.reflux_fine + ((long long)e * 6 + 2 * d + side) * 4;
                if (fs[0] < 0) continue;
                const T dx = T(g.dx[lev][d]);
                for (int t = threadIdx.x; t < TRANS; t += blockDim.x) {
                    const int th = D == 3 ? t / N : 0;       // transverse (hi, lo) in (z, y, x) order
                    const int tl = D == 1 ? 0 : (D == 3 ? t % N : t);
                    int cell[3] = {0, 0, 0};
                    cell[d] = side ? N - 1 : 0;
                    {
                        int j = 0;
                        for (int e2 = D - 1; e2 >= 0; --e2) {   // hi transverse first
                            if (e2 == d) continue;
                            cell[e2] = (D == 3 && j == 0) ? th : tl;
                            ++j;
                        }
                    }
                    const int sx = cell[0] + G, sy = D >= 2 ? cell[1] + G : 0, sz = D == 3 ? cell[2] + G : 0;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        T acc = T(0);
                        bool first = true;
                        for (int ah = 0; ah < (D == 3 ? 2 : 1); ++ah) {
                            for (int al = 0; al < (D >= 2 ? 2 : 1); ++al) {
                                const int fh = 2 * th + ah, fl = 2 * tl + al;
                                const int ph = fh / N, pl = fl / N;
                                const int lh = fh % N, ll = fl % N;
                                const int fslot = D == 3 ? fs[ph * 2 + pl] : (D == 2 ? fs[pl] : fs[0]);
                                const int fidx = D == 3 ? lh * N + ll : (D == 2 ? ll : 0);
                                if (fslot < 0) {             // inconsistent table: report, skip
                                    atomicOr(&g.time->err, ERR_MESH);
                                    continue;
                                }
                                const T val = faces[((long long)fslot * 2 * D + 2 * d + (1 - side)) * NV * TRANS +
                                                    v * TRANS + fidx];
                                acc = first ? val : acc + val;
                                first = false;
                            }
                        }
                        const T Ff = acc * T(D == 3 ? 0.25 : (D == 2 ? 0.5 : 1.0));
                        const T Fc = faces[((long long)slot * 2 * D + 2 * d + side) * NV * TRANS + v * TRANS + t];
                        const T diff = Num<T>::div(Ff - Fc, dx);
                        const long long id = slot_index(g, slot, v, sz, sy, sx);
                        const T u = Uout[id];
                        Uout[id] = side ? u - rb * (dt * diff) : u + rb * (dt * diff);
                    }
                }
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K6: restriction of level `level` into its parents: the covered coarse cell
// takes (sum of its 2^d children in lexicographic z, y, x order) * 2^-d,
// summed in FP64 (FP32 fields: an error-free FP32 pair sum, rounded once)
// ---------------------------------------------------------------------------
template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_restrict(Grid g, T* U, int level, int one_slot) {
    // thread <-> CP coarse cells adjacent in x (FP32: 2, FP64: 1), whose
    // children of each (y, z) offset are VE consecutive fine cells of a row:
    // one aligned 16-byte vector (interior rows start on a 32-byte boundary)
    constexpr int NV = D + 2;
    constexpr int VE = 16 / (int)sizeof(T);
    constexpr int CP = VE / 2;
    constexpr int H = N / 2;
    constexpr int HC = (D == 1 ? H : (D == 2 ? H * H : H * H * H)) / CP;
    constexpr int NYZ = 1 << (D - 1);                    // child (y, z) offsets
    constexpr int NCH = 1 << D;
    if (g.time->cancel) return;                          // a void step (see DevTime::cancel)
    const int lo = g.level_off[level], hi = g.level_off[level + 1];
    const int npatch = one_slot >= 0 ? 1 : hi - lo;
    const long long total = (long long)npatch * HC;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(it / HC);
        const int ci = (int)(it - (long long)pi * HC);
        const int slot = one_slot >= 0 ? one_slot : g.all_list[lo + pi];
        const int par = g.parent[slot];
        if (par < 0) {
            atomicOr(&g.time->err, ERR_MESH);
            continue;
        }
        constexpr int HX = H / CP;
        const int cx = (ci % HX) * CP, cy = D >= 2 ? (ci / HX) % H : 0, cz = D == 3 ? ci / (HX * H) : 0;
        const int ox = (g.coord[slot * 3 + 0] & 1) * H, oy = D >= 2 ? (g.coord[slot * 3 + 1] & 1) * H : 0,
                  oz = D == 3 ? (g.coord[slot * 3 + 2] & 1) * H : 0;
        T f[NV][NYZ][VE];                                  // [var][(az, ay)][fine x]
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int k = 0; k < NYZ; ++k) {
                const int ay = D >= 2 ? k & 1 : 0, az = D == 3 ? k >> 1 : 0;
                Vec16<T>::load(U + slot_index(g, slot, v, D == 3 ? 2 * cz + az + G : 0, D >= 2 ? 2 * cy + ay + G : 0,
                                              2 * cx + G),
                               f[v][k]);
            }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int q = 0; q < CP; ++q) {
                // the coarse cell's children in lexicographic z, y, x order
                T ch[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) ch[k] = f[v][k >> 1][2 * q + (k & 1)];
                const T mean = restrict_mean<T, D>(ch);
                U[slot_index(g, par, v, D == 3 ? oz + cz + G : 0, D >= 2 ? oy + cy + G : 0, ox + cx + q + G)] = mean;
            }
    }
}

// ---------------------------------------------------------------------------
// K7: CFL reduction over leaf cells: lambda = sum_d (|u_d| + c) / dx_d in FP64,
// c = sqrt(gamma p / rho); block max by warp shuffles, grid max by atomicMax
// on the bit pattern (valid for non-negative doubles)
// ---------------------------------------------------------------------------
template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_cfl(Grid g, const T* U, int one_slot) {
    // the running maximum is kept in the storage precision (exact: the
    // maximum of FP32 values converts to the maximum of their FP64 images)
    // and turned into FP64 once per CTA. A work item is VE consecutive
    // interior cells of a row, read as one aligned 16-byte vector per
    // variable (interior rows start on a 32-byte boundary)
    constexpr int NV = D + 2;
    constexpr int VE = Vec16<T>::VE;
    constexpr int NC = (D == 1 ? N : (D == 2 ? N * N : N * N * N)) / VE;
    if (g.time->cancel) return;                          // a void step (see DevTime::cancel)
    const int npatch = one_slot >= 0 ? 1 : g.counts[1];
    const long long total = (long long)npatch * NC;
    const T gamma = T(g.gamma);
    const T gm1 = T(g.gamma) - T(1);
    T lmax = T(0);
    bool bad = false;
#pragma unroll 2
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total;
         it += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(it / NC);
        const int ci = (int)(it - (long long)pi * NC);
        const int slot = one_slot >= 0 ? one_slot : g.leaf_list[pi];
        const int lev = g.level[slot];
        const int x = (ci % (N / VE)) * VE, y = D >= 2 ? (ci / (N / VE)) % N : 0, z = D == 3 ? ci / ((N / VE) * N) : 0;
        T Uv[NV][VE];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            Vec16<T>::load(U + slot_index(g, slot, v, D == 3 ? z + G : 0, D >= 2 ? y + G : 0, x + G), Uv[v]);
        T idx[D];
#pragma unroll
        for (int d = 0; d < D; ++d) idx[d] = T(g.dx[lev][d]);
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            T Uc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Uc[v] = Uv[v][e];
            T rho, u[D], p, Tt;
            primitives<T, D>(Uc, gm1, rho, u, p, Tt);
            if (!(rho > T(0)) || !(p > T(0))) bad = true;
            const T c = Num<T>::sqr(Num<T>::div(gamma * p, rho));
            T lam = Num<T>::div(fabs(u[0]) + c, idx[0]);
#pragma unroll
            for (int d = 1; d < D; ++d) lam = lam + Num<T>::div(fabs(u[d]) + c, idx[d]);
            if (!((double)lam <= 1.0e300)) bad = true;       // FP32: not finite; FP64: out of range
            else lmax = lmax > lam ? lmax : lam;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T other = __shfl_xor_sync(0xffffffffu, lmax, o);
        lmax = lmax > other ? lmax : other;
    }
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = (double)lmax;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&g.time->err, ERR_NONFINITE);
    if (wid == 0) {
        double m = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&g.time->lam, (unsigned long long)__double_as_longlong(m));
    }
}

// ---------------------------------------------------------------------------
// K9 (plain): relative-jump sensor on rho and p over the band [-2, N+1]^d of
// each leaf patch (in-domain cells): a cell is flagged if for some dimension
// |phi+ - phi-| > theta (phi+ + 2 phi0 + phi-) for phi in (rho, p) (the
// relative jump above theta, without the division). A work item is a patch
// (1D/2D) or a slab of DZB band planes of it (3D, four slabs); rho and p of
// the slab and its +-1 planes are staged in shared memory in the storage
// precision from 16-byte vector loads of the slot rows, and a patch's flag is
// the OR over its items.
// ---------------------------------------------------------------------------
template <typename T, int D, int N> struct FlagStage {
    static constexpr int S = N + 2 * G;
    static constexpr int XP = PatchShape<T, N>::XP;          // pad before the first ghost of a row
    // staged rows: the aligned 16-byte vectors of the slot row that cover
    // slot x in [0, S), from vector XV0 on; staged x = slot x + XO
    static constexpr int VE = 16 / (int)sizeof(T);
    static constexpr int XV0 = XP / VE;
    static constexpr int NXV = (XP + S + VE - 1) / VE - XV0;
    static constexpr int SXP = NXV * VE;                     // x pitch of the staged rows
    static constexpr int XO = XP - XV0 * VE;
    static constexpr int B = N + 4;                         // band cells per dimension
    static constexpr int NSLAB = D == 3 ? 4 : 1;
    static constexpr int DZB = D == 3 ? B / 4 : 1;           // band planes per slab
    static_assert(D != 3 || B % 4 == 0, "four slabs tile the band");
    static constexpr int PZ = D == 3 ? DZB + 2 : 1;          // staged planes
    static constexpr int SY = D >= 2 ? S : 1;
    static constexpr int NS = PZ * SY * SXP;                 // staged cells per field
};

template <typename T, int D, int N>
constexpr size_t flag_smem_bytes() { return 2 * sizeof(T) * FlagStage<T, D, N>::NS; }

template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_flag_plain(Grid g, const T* U, int* anyflag) {
    using F = FlagStage<T, D, N>;
    constexpr int NV = D + 2;
    constexpr int B = F::B;
    constexpr int NB = D == 1 ? B : (D == 2 ? B * B : B * B * F::DZB);     // band cells per item
    constexpr int VE = F::VE, NXV = F::NXV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* srho = reinterpret_cast<T*>(smem_raw);
    T* sp = srho + F::NS;
    const int npatch = g.counts[1];
    const T gm1 = T(g.gamma) - T(1);
    const T thr = T(g.theta_rho), thp = T(g.theta_p);
    for (int item = blockIdx.x; item < npatch * F::NSLAB; item += gridDim.x) {
        const int pi = item / F::NSLAB, slab = item - pi * F::NSLAB;
        const int slot = g.leaf_list[pi];
        const int lev = g.level[slot];
        const int c[3] = {g.coord[slot * 3], g.coord[slot * 3 + 1], g.coord[slot * 3 + 2]};
        const int sz0 = D == 3 ? slab * F::DZB : 0;             // first staged slot plane
        for (int iv = threadIdx.x; iv < F::PZ * F::SY * NXV; iv += blockDim.x) {
            const int xv = iv % NXV, y = (iv / NXV) % F::SY, z = iv / (NXV * F::SY);
            T Uv[NV][VE];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T* src = U + slot_index(g, slot, v, sz0 + z, y, xv * VE - F::XO);   // aligned
                if constexpr (sizeof(T) == 4) {
                    const float4 q = *reinterpret_cast<const float4*>(src);
                    Uv[v][0] = q.x; Uv[v][1] = q.y; Uv[v][2] = q.z; Uv[v][3] = q.w;
                } else {
                    const double2 q = *reinterpret_cast<const double2*>(src);
                    Uv[v][0] = q.x; Uv[v][1] = q.y;
                }
            }
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                T Uc[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) Uc[v] = Uv[v][e];
                T rho, u[D], p, Tt;
                primitives<T, D>(Uc, gm1, rho, u, p, Tt);
                const int idx = (z * F::SY + y) * F::SXP + xv * VE + e;
                srho[idx] = rho;
                sp[idx] = p;
            }
        }
        __syncthreads();
        bool any = false;
        for (int bi = threadIdx.x; bi < NB; bi += blockDim.x) {
            const int l[3] = {bi % B - 2, D >= 2 ? (bi / B) % B - 2 : 0,
                              D == 3 ? bi / (B * B) - 2 + slab * F::DZB : 0};
            bool indom = true;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                if (g.periodic[d]) continue;
                const int Gd = c[d] * N + l[d];
                indom = indom && Gd >= 0 && Gd < g.ext[lev][d] * N;
            }
            if (!indom) continue;
            const int i0 = ((D == 3 ? l[2] + G - sz0 : 0) * F::SY + sc<D>(1, l[1])) * F::SXP + sc<D>(0, l[0]) + F::XO;
            const T r0 = srho[i0], p0 = sp[i0];
            bool f = false;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int st = d == 0 ? 1 : (d == 1 ? F::SXP : F::SXP * F::SY);
                const T rm = srho[i0 - st], rp = srho[i0 + st];
                const T pm = sp[i0 - st], pp = sp[i0 + st];
                f = f || (fabs(rp - rm) > thr * (rp + T(2) * r0 + rm)) || (fabs(pp - pm) > thp * (pp + T(2) * p0 + pm));
            }
            any = any || f;
        }
        const int res = __syncthreads_or(any);
        if (threadIdx.x == 0 && res) atomicOr(&anyflag[slot], 3);   // refine and keep
    }
}

// ---------------------------------------------------------------------------
// K13: initial conditions point-sampled at cell centres (FP64, then stored)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double splitmix_unit(unsigned long long seed, unsigned long long n) {
    // output n+1 of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014), 53-bit mantissa
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

template <int D>
__device__ void ic_primitive(const Grid& g, const double* X, const int* Gi, int lev, const double* pre,
                             const double* post, double& rho, double* u, double& p) {
    const double x = X[0];
    for (int d = 0; d < 3; ++d) u[d] = 0.0;
    switch (g.ic) {
    case AMR_IC_SOD: {
        const bool left = x < 0.5;
        rho = left ? 1.0 : 0.125;
        p = left ? 1.0 : 0.1;
    } break;
    case AMR_IC_SHU_OSHER: {
        const bool left = x < -4.0;
        rho = left ? 3.857143 : 1.0 + 0.2 * sin(5.0 * x);
        u[0] = left ? 2.629369 : 0.0;
        p = left ? 10.33333 : 1.0;
    } break;
    case AMR_IC_RIEMANN2D: {
        const bool east = x > 0.5, north = X[1] > 0.5;
        if (east && north) { rho = 1.5; u[0] = 0.0; u[1] = 0.0; p = 1.5; }
        else if (!east && north) { rho = 0.5323; u[0] = 1.206; u[1] = 0.0; p = 0.3; }
        else if (!east && !north) { rho = 0.138; u[0] = 1.206; u[1] = 1.206; p = 0.029; }
        else { rho = 0.5323; u[0] = 0.0; u[1] = 1.206; p = 0.3; }
    } break;
    case AMR_IC_DMR: {
        const bool behind = x < 1.0 / 6.0 + X[1] / sqrt(3.0);
        const double* st = behind ? post : pre;
        rho = st[0]; u[0] = st[1]; u[1] = st[2]; p = st[3];
    } break;
    case AMR_IC_BLAST3D: {
        const double dxc = X[0] - 0.5, dyc = X[1] - 0.5, dzc = X[2] - 0.5;
        const double r2 = dxc * dxc + dyc * dyc + dzc * dzc;
        p = r2 < 0.01 ? 100.0 : 0.1;
        const long long ib0 = Gi[0] >> lev, ib1 = Gi[1] >> lev, ib2 = Gi[2] >> lev;
        const long long lin = (ib2 * g.base_cells[1] + ib1) * g.base_cells[0] + ib0;
        const double xi = splitmix_unit(g.seed, (unsigned long long)lin);
        rho = 1.0 + g.amp * (2.0 * xi - 1.0);
    } break;
    case AMR_IC_IMPLOSION: {
        const bool inside = fabs(X[0]) + fabs(X[1]) < 0.15;
        rho = inside ? 0.125 : 1.0;
        p = inside ? 0.140 : 1.0;
    } break;
    case AMR_IC_DENSITY_WAVE: {
        rho = 1.0 + 0.2 * sin(2.0 * 3.141592653589793 * x);
        u[0] = 1.0;
        p = 1.0;
    } break;
    case AMR_IC_SHEAR_LAYER: {
        const double y = X[1];
        const double c1 = sqrt(g.gamma * 1.0 / 1.0), c2 = sqrt(g.gamma * 1.0 / 2.0);
        const double du = 0.7 * (c1 + c2);
        const double f = 0.5 * (tanh((y + 0.15) / 0.01) - tanh((y - 0.15) / 0.01));
        rho = 2.0 + (1.0 - 2.0) * f;
        u[0] = -0.5 * du + du * f;
        const double a = (y - 0.15) / 0.02, b = (y + 0.15) / 0.02;
        u[1] = 0.05 * sin(2.0 * 3.141592653589793 * 5.0 * (x + 0.3) / 0.6) * (exp(-(a * a)) + exp(-(b * b)));
        p = 1.0;
    } break;
    default: {   // AMR_IC_CONSTANT
        rho = 1.0; p = 1.0;
        u[0] = 0.3; u[1] = -0.2; u[2] = 0.1;
    } break;
    }
}

template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_init_ic(Grid g, T* U, const int* list, int n, double4 pre4, double4 post4) {
    constexpr int NC = D == 1 ? N : (D == 2 ? N * N : N * N * N);
    const double pre[4] = {pre4.x, pre4.y, pre4.z, pre4.w};
    const double post[4] = {post4.x, post4.y, post4.z, post4.w};
    const double gm1 = g.gamma - 1.0;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < (long long)n * NC;
         it += (long long)gridDim.x * blockDim.x) {
        const int pi = (int)(it / NC);
        const int ci = (int)(it - (long long)pi * NC);
        const int slot = list[pi];
        const int lev = g.level[slot];
        const int l[3] = {ci % N, D >= 2 ? (ci / N) % N : 0, D == 3 ? ci / (N * N) : 0};
        int Gi[3];
        double X[3];
        for (int d = 0; d < 3; ++d) {
            Gi[d] = d < D ? g.coord[slot * 3 + d] * N + l[d] : 0;
            X[d] = g.lo[d] + ((double)Gi[d] + 0.5) * g.dx[lev][d];
        }
        double rho, u[3], p;
        ic_primitive<D>(g, X, Gi, lev, pre, post, rho, u, p);
        double usq = u[0] * u[0];
        for (int d = 1; d < D; ++d) usq = usq + u[d] * u[d];
        const int sx = l[0] + G, sy = D >= 2 ? l[1] + G : 0, sz = D == 3 ? l[2] + G : 0;
        U[slot_index(g, slot, 0, sz, sy, sx)] = T(rho);
        for (int d = 0; d < D; ++d) U[slot_index(g, slot, 1 + d, sz, sy, sx)] = T(rho * u[d]);
        U[slot_index(g, slot, D + 1, sz, sy, sx)] = T(p / gm1 + 0.5 * rho * usq);
    }
}

// K12: interiors of new patches by prolongation from their parents (one CTA per patch)
template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_prolong_new(Grid g, T* U, const int* list, int n) {
    constexpr int NV = D + 2;
    constexpr int NC = D == 1 ? N : (D == 2 ? N * N : N * N * N);
    __shared__ PatchMeta m;
    for (int pi = blockIdx.x; pi < n; pi += gridDim.x) {
        const int slot = list[pi];
        load_meta(g, slot, m);
        for (int ci = threadIdx.x; ci < NC; ci += blockDim.x) {
            int l[3] = {ci % N, D >= 2 ? (ci / N) % N : 0, D == 3 ? ci / (N * N) : 0};
            T val[NV];
            prolong_cell<T, D, N, false>(g, U, m, l, val);
            const int sx = l[0] + G, sy = D >= 2 ? l[1] + G : 0, sz = D == 3 ? l[2] + G : 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) U[slot_index(g, slot, v, sz, sy, sx)] = val[v];
        }
        __syncthreads();
    }
}

// K8: conservation sums over leaf cells (per-patch partials, then a fixed-order total)
template <typename T, int D, int N>
__global__ void __launch_bounds__(256) k_cons_partial(Grid g, const T* U, double* partial) {
    constexpr int NV = D + 2;
    constexpr int NC = D == 1 ? N : (D == 2 ? N * N : N * N * N);
    __shared__ double red[NV][256];
    const int npatch = g.counts[1];
    for (int pi = blockIdx.x; pi < npatch; pi += gridDim.x) {
        const int slot = g.leaf_list[pi];
        double acc[NV];
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
        for (int ci = threadIdx.x; ci < NC; ci += blockDim.x) {
            const int x = ci % N, y = D >= 2 ? (ci / N) % N : 0, z = D == 3 ? ci / (N * N) : 0;
            for (int v = 0; v < NV; ++v)
                acc[v] += (double)U[slot_index(g, slot, v, D == 3 ? z + G : 0, D >= 2 ? y + G : 0, x + G)];
        }
        for (int v = 0; v < NV; ++v) red[v][threadIdx.x] = acc[v];
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s)
                for (int v = 0; v < NV; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x < NV) {
            const int lev = g.level[slot];
            double vol = 1.0;
            for (int d = 0; d < D; ++d) vol *= g.dx[lev][d];
            partial[(long long)pi * NV + threadIdx.x] = red[threadIdx.x][0] * vol;
        }
        __syncthreads();
    }
}

template <int NV>
__global__ void k_cons_total(const int* counts, const double* partial, double* out) {
    __shared__ double red[NV][256];
    const int n = counts[1];
    double acc[NV];
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int v = 0; v < NV; ++v) acc[v] += partial[(long long)i * NV + v];
    for (int v = 0; v < NV; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int v = 0; v < NV; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < NV) out[threadIdx.x] = red[threadIdx.x][0];
}

// dense interiors <-> pool
template <typename T, int D, int N>
__global__ void k_unpack(Grid g, const T* U, const int* slots, int n, double* out) {
    constexpr int NV = D + 2;
    constexpr int NC = D == 1 ? N : (D == 2 ? N * N : N * N * N);
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < (long long)n * NV * NC;
         it += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(it % NC);
        const int v = (int)((it / NC) % NV);
        const int pi = (int)(it / ((long long)NC * NV));
        const int x = ci % N, y = D >= 2 ? (ci / N) % N : 0, z = D == 3 ? ci / (N * N) : 0;
        out[it] = (double)U[slot_index(g, slots[pi], v, D == 3 ? z + G : 0, D >= 2 ? y + G : 0, x + G)];
    }
}

template <typename T, int D, int N>
__global__ void k_pack(Grid g, T* U, const int* slots, int n, const double* in) {
    constexpr int NV = D + 2;
    constexpr int NC = D == 1 ? N : (D == 2 ? N * N : N * N * N);
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < (long long)n * NV * NC;
         it += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(it % NC);
        const int v = (int)((it / NC) % NV);
        const int pi = (int)(it / ((long long)NC * NV));
        const int x = ci % N, y = D >= 2 ? (ci / N) % N : 0, z = D == 3 ? ci / (N * N) : 0;
        U[slot_index(g, slots[pi], v, D == 3 ? z + G : 0, D >= 2 ? y + G : 0, x + G)] = T(in[it]);
    }
}

}  // namespace amr
