// K1: Mooney-Rivlin nodal forces of every tet (Sec. 2, Sec. 3.1-3.2), one
// thread per tet, and the energy V_0 U per tet (K7, test support).
//
// Per tet, with vertex 4 (corner 3) as the origin of the local coordinates:
//   A_ik = u_i^k - u_i^4,  H = A B  (so F = I + H, Sec. 3.2),
//   P = dU/dF from the chain rule of Sec. 3.1 over the derivative table of
//       Sec. 3.2, which sums to
//       P = alpha F + beta cof(F) + gamma F C,
//       alpha = mu1 J^-2/3 + mu2 T_C J^-4/3,
//       beta  = -(mu1/3) T_C J^-5/3 - (mu2/3)(T_C^2 - T_C2) J^-7/3 + kappa (J-1),
//       gamma = -mu2 J^-4/3,  cof(F) = J F^-T,
//   f^a_i = -V_0 sum_l P_il B_al (a = 1..3), f^4 = -(f^1 + f^2 + f^3).
//
// FP32 without cancellation: at small strain the three terms of P are O(mu)
// each and cancel to O(mu |H|). Writing F = I + H, C = I + E (E = H + H^T +
// H^T H), cof(F) = (1 + tr H) I - H^T + cof(H) and F C = I + H + E + H E, the
// O(mu) parts collect into sigma I with
//   sigma = alpha + beta + gamma
//         = mu1 s (3j - e)/(3J) + mu2 s^2 (6j - e + 3je - e^2 + q)/(3J) + kappa j,
// where j = J - 1 = tr H + ((tr H)^2 - tr H^2)/2 + det H, e = tr E, q = tr E^2
// and s = J^-2/3 = exp(-2/3 log1p(j)). Every remaining term is O(|H|), so the
// result keeps FP32 relative accuracy down to the rest state.
#include "internal.cuh"

namespace cf {

__device__ __forceinline__ float det3(const float (&h)[3][3]) {
    return h[0][0] * (h[1][1] * h[2][2] - h[1][2] * h[2][1]) - h[0][1] * (h[1][0] * h[2][2] - h[1][2] * h[2][0]) +
           h[0][2] * (h[1][0] * h[2][1] - h[1][1] * h[2][0]);
}

// H = A B for tet t: A_ik = u_i^k - u_i^4 (Sec. 3.2), B = J^-1 precomputed.
__device__ __forceinline__ void tet_H(const MeshView &m, const float4 *__restrict__ u, int t, float (&H)[3][3]) {
    const int4 a = __ldg(m.tet + t);
    const float4 u0 = __ldg(u + a.x), u1 = __ldg(u + a.y), u2 = __ldg(u + a.z), u3 = __ldg(u + a.w);
    const float A[3][3] = {{u0.x - u3.x, u1.x - u3.x, u2.x - u3.x},
                           {u0.y - u3.y, u1.y - u3.y, u2.y - u3.y},
                           {u0.z - u3.z, u1.z - u3.z, u2.z - u3.z}};
    float B[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) B[k][j] = __ldg(m.B + (3 * k + j) * m.T + t);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[i][j] = A[i][0] * B[0][j] + A[i][1] * B[1][j] + A[i][2] * B[2][j];
}

// Invariant pieces shared by force and energy.
struct Inv {
    float t, e, q, j, J, L;  // tr H, tr E, tr E^2, J-1, J, log J
    float E[3][3];
};

__device__ __forceinline__ void invariants(const float (&H)[3][3], Inv &v) {
    v.t = H[0][0] + H[1][1] + H[2][2];
    float trH2 = 0.f, hh = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            trH2 += H[i][k] * H[k][i];
            hh += H[i][k] * H[i][k];
        }
    // E = H + H^T + H^T H (= C - I)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l)
            v.E[k][l] = H[k][l] + H[l][k] + H[0][k] * H[0][l] + H[1][k] * H[1][l] + H[2][k] * H[2][l];
    v.e = 2.f * v.t + hh;
    float q = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) q += v.E[k][l] * v.E[k][l];
    v.q = q;
    v.j = v.t + 0.5f * (v.t * v.t - trH2) + det3(H);
    v.J = 1.f + v.j;
    v.L = log1pf(v.j);
}

__global__ void __launch_bounds__(256) k_tet_force(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                   int tet_blocks, const float4 *__restrict__ u_prev,
                                                   float *__restrict__ F, LbmParams lp) {
    if ((int)blockIdx.x >= tet_blocks) {
        // Zero the force field on the delta support of x + u_prev: every
        // nonzero entry of F was spread there in the previous step.
        const int v = (blockIdx.x - tet_blocks) * blockDim.x + threadIdx.x;
        if (v >= m.V) return;
        Support sp;
        if (!support_of(m.origin, __ldg(m.xr + v), __ldg(u_prev + v), lp.ny, sp)) return;  // nothing was spread
        const int N = (int)lp.N;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const int Z = wrapi(sp.bz + dz, lp.nz);
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int n = wrapi(sp.bx + dx, lp.nx) + lp.nx * (sp.by + dy + lp.ny * Z);
                    F[n] = 0.f;
                    F[N + n] = 0.f;
                    F[2 * N + n] = 0.f;
                }
        }
        return;
    }
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;

    float H[3][3];
    tet_H(m, u, t, H);
    Inv v;
    invariants(H, v);
    if (!(v.J > 0.f)) atomicOr(err, ERR_INVERTED);

    const int c = __ldg(m.tcell + t);
    const float4 mat = __ldg(m.mat + c);
    const float mu1 = mat.x, mu2 = mat.y, kappa = mat.z;

    const float s = expf(-(2.f / 3.f) * v.L);  // J^-2/3
    const float s2 = s * s;                     // J^-4/3
    const float TC = 3.f + v.e;
    const float TC2 = 3.f + 2.f * v.e + v.q;
    const float iJ3 = 1.f / (3.f * v.J);
    const float alpha = mu1 * s + mu2 * TC * s2;
    const float beta = -(mu1 * TC * s + mu2 * (TC * TC - TC2) * s2) * iJ3 + kappa * v.j;
    const float gamma = -mu2 * s2;
    const float sigma = mu1 * s * (3.f * v.j - v.e) * iJ3 +
                        mu2 * s2 * (6.f * v.j - v.e + 3.f * v.j * v.e - v.e * v.e + v.q) * iJ3 + kappa * v.j;

    // cof(H)_il = dual of H: cofactor matrix
    float cofH[3][3];
    cofH[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
    cofH[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
    cofH[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
    cofH[1][0] = H[0][2] * H[2][1] - H[0][1] * H[2][2];
    cofH[1][1] = H[0][0] * H[2][2] - H[0][2] * H[2][0];
    cofH[1][2] = H[0][1] * H[2][0] - H[0][0] * H[2][1];
    cofH[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
    cofH[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
    cofH[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];

    float P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const float HE = H[i][0] * v.E[0][l] + H[i][1] * v.E[1][l] + H[i][2] * v.E[2][l];
            float p = alpha * H[i][l] + beta * (cofH[i][l] - H[l][i]) + gamma * (H[i][l] + v.E[i][l] + HE);
            if (i == l) p += sigma + beta * v.t;
            P[i][l] = p;
        }

    const float V0 = __ldg(m.V0 + t);
    float Bm[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bm[k][j] = __ldg(m.B + (3 * k + j) * m.T + t);
    float f[4][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            f[a][i] = -V0 * (P[i][0] * Bm[a][0] + P[i][1] * Bm[a][1] + P[i][2] * Bm[a][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) f[3][i] = -(f[0][i] + f[1][i] + f[2][i]);
#pragma unroll
    for (int a = 0; a < 4; ++a) m.fc[a * m.T + t] = make_float4(f[a][0], f[a][1], f[a][2], 0.f);
}

cudaError_t launch_tet_force(const MeshView &m, const float4 *u, unsigned *err, const float4 *u_prev, float *F,
                             const LbmParams *lp, cudaStream_t s) {
    if (m.T == 0) return cudaSuccess;
    const int bs = 64;  // ~20k tets: enough blocks for every SM
    const int tb = (m.T + bs - 1) / bs;
    const int cb = (u_prev && F && lp) ? (m.V + bs - 1) / bs : 0;
    LbmParams p{};
    if (lp) p = *lp;
    k_tet_force<<<tb + cb, bs, 0, s>>>(m, u, err, tb, u_prev, F, p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- energy
// U = mu1/2 (I-3) + mu2/2 (K-3) + kappa/2 (J-1)^2 (Sec. 2) with
// I - 3 = 3(s-1) + e s and K - 3 = 3(s^2-1) + (4e + e^2 - q) s^2 / 2.
__global__ void __launch_bounds__(256) k_energy(MeshView m, const float4 *__restrict__ u, int t0, int t1,
                                                double *partial) {
    __shared__ double red[256];
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    double e_t = 0.0;
    if (t < t1) {
        float H[3][3];
        tet_H(m, u, t, H);
        Inv v;
        invariants(H, v);
        const int c = __ldg(m.tcell + t);
        const float4 mat = __ldg(m.mat + c);
        const float sm1 = expm1f(-(2.f / 3.f) * v.L);
        const float s2m1 = expm1f(-(4.f / 3.f) * v.L);
        const float s = 1.f + sm1, s2 = 1.f + s2m1;
        const float Im3 = 3.f * sm1 + v.e * s;
        const float Km3 = 3.f * s2m1 + 0.5f * (4.f * v.e + v.e * v.e - v.q) * s2;
        const float U = 0.5f * mat.x * Im3 + 0.5f * mat.y * Km3 + 0.5f * mat.z * v.j * v.j;
        e_t = (double)__ldg(m.V0 + t) * (double)U;
    }
    red[threadIdx.x] = e_t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double *partial, int n, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        *out = s;
    }
}

cudaError_t launch_energy(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s) {
    const int nb = (t1 - t0 + 255) / 256;
    if (nb > 0) k_energy<<<nb, 256, 0, s>>>(m, u, t0, t1, partial);
    k_sum_partials<<<1, 32, 0, s>>>(partial, nb, out);
    return cudaGetLastError();
}

}  // namespace cf
