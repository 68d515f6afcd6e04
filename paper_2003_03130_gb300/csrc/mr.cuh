// Mooney-Rivlin first Piola stress P = dU/dF of one tet (Sec. 2, Sec. 3.1-3.2),
// shared by the force kernel (scalar S = float) and its forward-mode
// derivative (S = Dual: value and directional derivative), which the adjoint
// uses for Hessian-vector products.
//
// With H = A B (F = I + H), the chain rule of Sec. 3.1 over the derivative
// table of Sec. 3.2 sums to P = alpha F + beta cof(F) + gamma F C with
//   alpha = mu1 J^-2/3 + mu2 T_C J^-4/3,
//   beta  = -(mu1/3) T_C J^-5/3 - (mu2/3)(T_C^2 - T_C2) J^-7/3 + kappa (J-1),
//   gamma = -mu2 J^-4/3,  cof(F) = J F^-T.
// FP32 without cancellation: at small strain the three terms are O(mu) each
// and cancel to O(mu |H|). Writing C = I + E (E = H + H^T + H^T H),
// cof(F) = (1 + tr H) I - H^T + cof(H) and F C = I + H + E + H E, the O(mu)
// parts collect into sigma I with
//   sigma = alpha + beta + gamma
//         = mu1 s (3j - e)/(3J) + mu2 s^2 (6j - e + 3je - e^2 + q)/(3J) + kappa j,
// where j = J - 1 = tr H + ((tr H)^2 - tr H^2)/2 + det H, e = tr E, q = tr E^2
// and s = J^-2/3 = exp(-2/3 log1p(j)). Every remaining term is O(|H|).
#pragma once

#include "internal.cuh"

namespace cf {

// ---------------------------------------------------------------- dual numbers
struct Dual {
    float v, d;
    Dual() = default;
    __device__ __forceinline__ Dual(float a) : v(a), d(0.f) {}
    __device__ __forceinline__ Dual(float a, float b) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, fmaf(a.d, b.v, a.v * b.d)}; }
__device__ __forceinline__ Dual operator+(Dual a, float b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(float a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, float b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(float a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, float b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(float a, Dual b) { return {a * b.v, a * b.d}; }

__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ float val(Dual a) { return a.v; }
__device__ __forceinline__ float m_log1p(float a) { return log1pf(a); }
__device__ __forceinline__ Dual m_log1p(Dual a) { return {log1pf(a.v), a.d / (1.f + a.v)}; }
__device__ __forceinline__ float m_exp(float a) { return expf(a); }
__device__ __forceinline__ Dual m_exp(Dual a) {
    const float e = expf(a.v);
    return {e, e * a.d};
}
__device__ __forceinline__ float m_rcp(float a) { return 1.f / a; }
__device__ __forceinline__ Dual m_rcp(Dual a) {
    const float r = 1.f / a.v;
    return {r, -a.d * r * r};
}

// ---------------------------------------------------------------- stress
template <class S>
struct InvT {
    S t, e, q, j, J, L;  // tr H, tr E, tr E^2, J-1, J, log J
    S E[3][3];
};

template <class S>
__device__ __forceinline__ S det3t(const S (&h)[3][3]) {
    return h[0][0] * (h[1][1] * h[2][2] - h[1][2] * h[2][1]) - h[0][1] * (h[1][0] * h[2][2] - h[1][2] * h[2][0]) +
           h[0][2] * (h[1][0] * h[2][1] - h[1][1] * h[2][0]);
}

template <class S>
__device__ __forceinline__ void invariants_t(const S (&H)[3][3], InvT<S> &v) {
    v.t = H[0][0] + H[1][1] + H[2][2];
    S trH2 = 0.f, hh = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            trH2 = trH2 + H[i][k] * H[k][i];
            hh = hh + H[i][k] * H[i][k];
        }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            v.E[k][l] = H[k][l] + H[l][k] + H[0][k] * H[0][l] + H[1][k] * H[1][l] + H[2][k] * H[2][l];
    v.e = 2.f * v.t + hh;
    S q = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) q = q + v.E[k][l] * v.E[k][l];
    v.q = q;
    v.j = v.t + 0.5f * (v.t * v.t - trH2) + det3t(H);
    v.J = 1.f + v.j;
    v.L = m_log1p(v.j);
}

// P = dU/dF for F = I + H, moduli (mu1, mu2, kappa) and the invariants v of
// H (invariants_t; the caller may replace j, J and L by a more accurate J - 1).
template <class S>
__device__ __forceinline__ void mr_stress_inv(const S (&H)[3][3], float mu1, float mu2, float kappa,
                                              const InvT<S> &v, S (&P)[3][3]) {
    const S s = m_exp(-(2.f / 3.f) * v.L);  // J^-2/3
    const S s2 = s * s;                     // J^-4/3
    const S TC = 3.f + v.e;
    const S TC2 = 3.f + 2.f * v.e + v.q;
    const S iJ3 = m_rcp(3.f * v.J);
    const S alpha = mu1 * s + mu2 * TC * s2;
    const S beta = kappa * v.j - (mu1 * TC * s + mu2 * (TC * TC - TC2) * s2) * iJ3;
    const S gamma = -mu2 * s2;
    const S sigma = mu1 * s * (3.f * v.j - v.e) * iJ3 +
                    mu2 * s2 * (6.f * v.j - v.e + 3.f * v.j * v.e - v.e * v.e + v.q) * iJ3 + kappa * v.j;
    S cofH[3][3];
    cofH[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
    cofH[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
    cofH[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
    cofH[1][0] = H[0][2] * H[2][1] - H[0][1] * H[2][2];
    cofH[1][1] = H[0][0] * H[2][2] - H[0][2] * H[2][0];
    cofH[1][2] = H[0][1] * H[2][0] - H[0][0] * H[2][1];
    cofH[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
    cofH[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
    cofH[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const S HE = H[i][0] * v.E[0][l] + H[i][1] * v.E[1][l] + H[i][2] * v.E[2][l];
            S p = alpha * H[i][l] + beta * (cofH[i][l] - H[l][i]) + gamma * (H[i][l] + v.E[i][l] + HE);
            if (i == l) p = p + sigma + beta * v.t;
            P[i][l] = p;
        }
}

// P = dU/dF for F = I + H and moduli (mu1, mu2, kappa); v gets the invariants.
template <class S>
__device__ __forceinline__ void mr_stress(const S (&H)[3][3], float mu1, float mu2, float kappa, InvT<S> &v,
                                          S (&P)[3][3]) {
    invariants_t(H, v);
    mr_stress_inv(H, mu1, mu2, kappa, v, P);
}

// Nearly incompressible tets (kappa >= kStiffVolume (mu1 + mu2), Poisson
// ratio 0.495 and above) take J - 1 in FP64. The volume term kappa (J - 1)
// multiplies any rounding of J - 1 by kappa: under a nearly isochoric
// deformation J - 1 is small against |H|, and J - 1 from the FP32 B and
// FP32 products carries errors of ~1e-7 |H|, which reach the forces
// amplified by kappa / mu (measured: 7e-5 relative at kappa = 2,000 mu in
// simple shear). In FP64, from the FP32 displacements (exact in FP64) and the
// FP64 B of the precompute, J - 1 is exact to ~1e-16 |H|; the rest of the
// stress stays FP32.
constexpr float kStiffVolume = 100.f;

__device__ __forceinline__ bool needs_fp64_volume(const MeshView &m, float4 mat) {
    return m.B64 != nullptr && mat.z >= kStiffVolume * (mat.x + mat.y);
}

// J - 1 = tr H + ((tr H)^2 - tr H^2) / 2 + det H in FP64 with H = A B, A from
// the column differences a_k = w_k - w_4 (k = 1..3, exact in FP64), B from
// B64 ([9][T]).
__device__ __forceinline__ double volume_change64_body(const double *__restrict__ B64, int T, int t, float4 w0,
                                                       float4 w1, float4 w2, float4 w3) {
    const double A[3][3] = {{(double)w0.x - w3.x, (double)w1.x - w3.x, (double)w2.x - w3.x},
                            {(double)w0.y - w3.y, (double)w1.y - w3.y, (double)w2.y - w3.y},
                            {(double)w0.z - w3.z, (double)w1.z - w3.z, (double)w2.z - w3.z}};
    double Bm[3][3], H[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bm[k][j] = __ldg(B64 + (size_t)(3 * k + j) * T + t);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[i][j] = A[i][0] * Bm[0][j] + A[i][1] * Bm[1][j] + A[i][2] * Bm[2][j];
    const double tr = H[0][0] + H[1][1] + H[2][2];
    double tr2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) tr2 += H[i][k] * H[k][i];
    const double det = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                       H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                       H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
    return tr + 0.5 * (tr * tr - tr2) + det;
}

// The same as a called function, for kernels whose FP32 path the FP64
// registers would otherwise crowd (one thread per tet).
static __device__ __noinline__ double volume_change64(const double *__restrict__ B64, int T, int t, float4 w0, float4 w1,
                                               float4 w2, float4 w3) {
    return volume_change64_body(B64, T, t, w0, w1, w2, w3);
}

// Replace J - 1 (and J, log J) of v by j.
__device__ __forceinline__ void set_volume_change(InvT<float> &v, float j) {
    v.j = j;
    v.J = 1.f + j;
    v.L = log1pf(j);
}

// Corner forces f^a_i = -V_0 sum_l P_il B_al (a = 1..3), f^4 = -(f^1 + f^2 + f^3)
// (Sec. 3.1 with dF_kl/du_i^a = delta_ki B_ml (delta_ma - delta_4a)).
__device__ __forceinline__ void corner_forces(const float (&P)[3][3], const float (&Bm)[3][3], float V0,
                                              float (&f)[4][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) f[a][i] = -V0 * (P[i][0] * Bm[a][0] + P[i][1] * Bm[a][1] + P[i][2] * Bm[a][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) f[3][i] = -(f[0][i] + f[1][i] + f[2][i]);
}

// A B for a tet: A_ik = w_i^k - w_i^4 from four per-vertex vectors.
__device__ __forceinline__ void tet_grad(const float4 &w0, const float4 &w1, const float4 &w2, const float4 &w3,
                                         const float (&Bm)[3][3], float (&H)[3][3]) {
    const float A[3][3] = {{w0.x - w3.x, w1.x - w3.x, w2.x - w3.x},
                           {w0.y - w3.y, w1.y - w3.y, w2.y - w3.y},
                           {w0.z - w3.z, w1.z - w3.z, w2.z - w3.z}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[i][j] = A[i][0] * Bm[0][j] + A[i][1] * Bm[1][j] + A[i][2] * Bm[2][j];
}

// Material slot of tet t.
__device__ __forceinline__ int mat_slot(const MeshView &m, int t) { return __ldg((m.tmat ? m.tmat : m.tcell) + t); }

// B, V0 and the tet's material slot: three 16-byte loads from the packed
// rows when the view has them, else eleven 4-byte loads from the separate
// arrays.
__device__ __forceinline__ void load_tet_params(const MeshView &m, int t, float (&Bm)[3][3], float &V0, int &slot) {
    if (m.Bp) {
        const float4 r0 = __ldg(m.Bp + t), r1 = __ldg(m.Bp + m.T + t), r2 = __ldg(m.Bp + 2 * m.T + t);
        Bm[0][0] = r0.x; Bm[0][1] = r0.y; Bm[0][2] = r0.z;
        Bm[1][0] = r1.x; Bm[1][1] = r1.y; Bm[1][2] = r1.z;
        Bm[2][0] = r2.x; Bm[2][1] = r2.y; Bm[2][2] = r2.z;
        V0 = r0.w;
        slot = __float_as_int(r1.w);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bm[k][j] = __ldg(m.B + (3 * k + j) * m.T + t);
    V0 = __ldg(m.V0 + t);
    slot = mat_slot(m, t);
}

__device__ __forceinline__ void load_B(const MeshView &m, int t, float (&Bm)[3][3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bm[k][j] = __ldg(m.B + (3 * k + j) * m.T + t);
}

}  // namespace cf
