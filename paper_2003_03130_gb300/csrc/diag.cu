// K8: Taylor deformation parameter of a cell on the device (Sec. 3.3).
//
// Inertia tensor of the tet mesh at the current positions,
//   Theta_ij = sum_l V_l (r^l.r^l delta_ij - r^l_i r^l_j),
// with r^l the centroid of tet l relative to the volume-weighted centroid of
// the cell and V_l its current volume. One pass accumulates, in double and in
// a fixed order (per-block tree, then the blocks in index order), the moments
// M = sum V, m = sum V c, S = sum V c c^T of the tet centroids c; then
// Theta = (tr S' ) I - S' with S' = S - m m^T / M. A single thread finishes:
// eigenvalues theta_1 >= theta_2 >= theta_3 by cyclic Jacobi rotations,
// semi-axes a_i = sqrt((5 / 2M)(...)) (the printed expression has units of
// length squared, so a_i is its square root), D = (a3 - a1)/(a3 + a1), and the
// inclination of the major axis (eigenvector of theta_3) to x in the x-y
// plane, in (-90, 90] degrees. Positions enter relative to the cell's integer
// origin (translation does not change Theta).
#include "internal.cuh"

namespace cf {

constexpr int kTaylorBlock = 256;
constexpr int kMoments = 10;  // M, m (3), S (6: xx yy zz xy xz yz)

__global__ void __launch_bounds__(kTaylorBlock) k_taylor_partial(MeshView m, const float4 *__restrict__ u, int t0,
                                                                 int t1, double *partial) {
    __shared__ double red[kMoments][kTaylorBlock];
    const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
    double v[kMoments] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (t < t1) {
        const int4 a = __ldg(m.tet + t);
        const int idx[4] = {a.x, a.y, a.z, a.w};
        double p[4][3];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 xr = __ldg(m.xr + idx[c]), du = __ldg(u + idx[c]);
            p[c][0] = (double)(xr.x + du.x);
            p[c][1] = (double)(xr.y + du.y);
            p[c][2] = (double)(xr.z + du.z);
        }
        double e[3][3];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) e[k][i] = p[k][i] - p[3][i];
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        const double V = fabs(det) / 6.0;
        double c[3];
        for (int i = 0; i < 3; ++i) c[i] = 0.25 * (p[0][i] + p[1][i] + p[2][i] + p[3][i]);
        v[0] = V;
        v[1] = V * c[0];
        v[2] = V * c[1];
        v[3] = V * c[2];
        v[4] = V * c[0] * c[0];
        v[5] = V * c[1] * c[1];
        v[6] = V * c[2] * c[2];
        v[7] = V * c[0] * c[1];
        v[8] = V * c[0] * c[2];
        v[9] = V * c[1] * c[2];
    }
#pragma unroll
    for (int k = 0; k < kMoments; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kTaylorBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < kMoments; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kMoments) partial[blockIdx.x * kMoments + threadIdx.x] = red[threadIdx.x][0];
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations; columns of
// V are the eigenvectors.
__device__ void jacobi3(double A[3][3], double V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-30 * (dia > 1.0 ? dia : 1.0)) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                // A <- R^T A R, V <- V R with R the rotation in the (p, q) plane
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
}

// out[10]: D, D from the printed (squared) expression, inclination (deg),
// a1 <= a2 <= a3, theta1 >= theta2 >= theta3, volume.
__global__ void k_taylor_final(const double *partial, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[kMoments] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < kMoments; ++k) s[k] += partial[b * kMoments + k];
    const double M = s[0];
    const double c0[3] = {s[1] / M, s[2] / M, s[3] / M};
    // second moments about the centroid
    double S[3][3];
    S[0][0] = s[4] - M * c0[0] * c0[0];
    S[1][1] = s[5] - M * c0[1] * c0[1];
    S[2][2] = s[6] - M * c0[2] * c0[2];
    S[0][1] = S[1][0] = s[7] - M * c0[0] * c0[1];
    S[0][2] = S[2][0] = s[8] - M * c0[0] * c0[2];
    S[1][2] = S[2][1] = s[9] - M * c0[1] * c0[2];
    const double tr = S[0][0] + S[1][1] + S[2][2];
    double A[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = (i == j ? tr : 0.0) - S[i][j];
    jacobi3(A, V);
    double lam[3] = {A[0][0], A[1][1], A[2][2]};
    int ord[3] = {0, 1, 2};  // descending eigenvalues
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (lam[ord[j]] > lam[ord[i]]) {
                const int tmp = ord[i];
                ord[i] = ord[j];
                ord[j] = tmp;
            }
    const double t1 = lam[ord[0]], t2 = lam[ord[1]], t3 = lam[ord[2]];
    const double pre = 5.0 / (2.0 * M);
    const double a1s = pre * (-t1 + t2 + t3), a2s = pre * (t1 - t2 + t3), a3s = pre * (t1 + t2 - t3);
    const double a1 = sqrt(a1s > 0 ? a1s : 0), a2 = sqrt(a2s > 0 ? a2s : 0), a3 = sqrt(a3s > 0 ? a3s : 0);
    const int k3 = ord[2];
    double ang = atan2(V[1][k3], V[0][k3]) * (180.0 / 3.14159265358979323846);
    if (ang <= -90.0) ang += 180.0;
    if (ang > 90.0) ang -= 180.0;
    out[0] = (a3 - a1) / (a3 + a1);
    out[1] = (a3s - a1s) / (a3s + a1s);
    out[2] = ang;
    out[3] = a1;
    out[4] = a2;
    out[5] = a3;
    out[6] = t1;
    out[7] = t2;
    out[8] = t3;
    out[9] = M;
}

cudaError_t launch_taylor(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s) {
    const int nb = (t1 - t0 + kTaylorBlock - 1) / kTaylorBlock;
    if (nb > 0) k_taylor_partial<<<nb, kTaylorBlock, 0, s>>>(m, u, t0, t1, partial);
    k_taylor_final<<<1, 32, 0, s>>>(partial, nb, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cell strain
// Largest distance between two vertices of a cell (the elongation d_max of
// the cell strain, Sec. 6.1), by brute force over all pairs. Block b holds
// vertex tile b and sweeps the tiles b, b+1, ... through shared memory, so
// every pair meets once; the squared distances are reduced by a maximum,
// which does not depend on the order, first per block, then across blocks by
// atomicMax on the bit pattern (non-negative floats order like their bits).
// Positions enter relative to the cell's integer origin.
constexpr int kExtentBlock = 256;

__global__ void __launch_bounds__(kExtentBlock) k_max_extent(MeshView m, const float4 *__restrict__ u, int v0,
                                                             int nv, unsigned *out) {
    __shared__ float3 tile[kExtentBlock];
    __shared__ float red[kExtentBlock];
    const int i = blockIdx.x * kExtentBlock + threadIdx.x;
    const bool live = i < nv;
    // a padding slot takes the cell's first vertex: its distances are real pairs
    auto pos = [&](int k) {
        const float4 xr = __ldg(m.xr + v0 + k), du = __ldg(u + v0 + k);
        return make_float3(xr.x + du.x, xr.y + du.y, xr.z + du.z);
    };
    const float3 yi = pos(live ? i : 0);
    float best = 0.f;
    for (int jt = blockIdx.x; jt * kExtentBlock < nv; ++jt) {
        const int j = jt * kExtentBlock + threadIdx.x;
        __syncthreads();
        tile[threadIdx.x] = pos(j < nv ? j : 0);
        __syncthreads();
        for (int k = 0; k < kExtentBlock; ++k) {
            const float dx = tile[k].x - yi.x, dy = tile[k].y - yi.y, dz = tile[k].z - yi.z;
            best = fmaxf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int w = kExtentBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, __float_as_uint(red[0]));
}

cudaError_t launch_max_extent(const MeshView &m, const float4 *u, int v0, int nv, unsigned *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), s);
    if (e != cudaSuccess || nv <= 0) return e;
    k_max_extent<<<(nv + kExtentBlock - 1) / kExtentBlock, kExtentBlock, 0, s>>>(m, u, v0, nv, out);
    return cudaGetLastError();
}

}  // namespace cf
