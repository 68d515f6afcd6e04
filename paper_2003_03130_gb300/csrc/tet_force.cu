// K1: Mooney-Rivlin nodal forces of every tet (Sec. 2, Sec. 3.1-3.2), one
// thread per tet, two tets per thread, or four lanes per tet (a launch-shape
// choice), and the energy V_0 U per tet (K7, test support). The stress
// evaluation (the cancellation-free form of the paper's chain rule) is in
// mr.cuh.
#include "cell_ops.cuh"

namespace cf {

// Region marking in the force launch: the first mark_blocks blocks run one
// thread per vertex, marking the next step's force region. They come first
// so that their short, latency-bound work runs under the tets' rather than
// after it.
__device__ __forceinline__ bool mark_block(const MeshView &m, const float4 *__restrict__ u, const LbmParams &lp,
                                           const RegionSlot &mark, int mark_blocks) {
    if ((int)blockIdx.x >= mark_blocks) return false;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < m.V) {
        if (lp.dw == 4)
            mark_vertex<4>(m, u, lp, v, mark);
        else
            mark_vertex<2>(m, u, lp, v, mark);
    }
    return true;
}

// Six blocks of 256 per SM (40 registers, a small spill): this latency-
// bound kernel gains more from the extra resident warps than the spill costs
// (tet forces of the 400-cell suspension 190.6 -> 178.5 us against 56
// registers and four blocks).
__global__ void __launch_bounds__(256, 6) k_tet_force(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                   int mark_blocks, LbmParams lp, RegionSlot mark) {
    if (mark_block(m, u, lp, mark, mark_blocks)) return;
    const int t = (blockIdx.x - mark_blocks) * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    tet_corner_forces(m, u, err, t);
}

// Two tets per thread, t and t + blockDim (coalesced either way): both tets'
// loads are issued before either is computed, doubling the bytes a thread
// has in flight in this latency-bound kernel.
__global__ void __launch_bounds__(256, 2) k_tet_force2(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                     int mark_blocks, LbmParams lp, RegionSlot mark) {
    if (mark_block(m, u, lp, mark, mark_blocks)) return;
    const int t0 = 2 * (blockIdx.x - mark_blocks) * blockDim.x + threadIdx.x, t1 = t0 + blockDim.x;
    if (t0 >= m.T) return;
    TetIn a, b;
    tet_load(m, u, t0, a);
    if (t1 < m.T) tet_load(m, u, t1, b);
    tet_forces_store(m, a, err, t0);
    if (t1 < m.T) tet_forces_store(m, b, err, t1);
}

// Four lanes per tet, lane k = corner k (for meshes too small to fill the
// GPU with one thread per tet): each lane loads one vertex index and one
// displacement, lanes 0-2 one packed row of B, lane 3 the material; the
// columns a_k = w_k - w_4 of A meet in H = A B = sum_k a_k (x) B_k by a
// two-step shuffle tree over the four lanes, every lane evaluates the stress
// of the tet, lane k < 3 computes f^k = -V0 P B_k and lane 3 the balance
// f^4 = -(f^1 + f^2 + f^3) from a second shuffle tree; each lane stores its
// corner. Every lane of a warp takes part in the shuffles (tets past the end
// compute on zeros and store nothing). Needs the packed rows (m.Bp).
__global__ void __launch_bounds__(256, 4) k_tet_force4(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                      int mark_blocks, LbmParams lp, RegionSlot mark) {
    constexpr unsigned kAll = 0xffffffffu;
    if (mark_block(m, u, lp, mark, mark_blocks)) return;
    const int g = (blockIdx.x - mark_blocks) * blockDim.x + threadIdx.x;
    const int t = g >> 2, k = g & 3, lead = (threadIdx.x & 31) & ~3;
    const bool live = t < m.T;
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f), b = w, mat = w;
    if (live) {
        const int vid = __ldg(reinterpret_cast<const int *>(m.tet) + 4 * (size_t)t + k);
        w = __ldg(u + vid);
        if (k < 3)
            b = __ldg(m.Bp + (size_t)k * m.T + t);
        else
            mat = __ldg(m.mat + mat_slot(m, t));
    }
    const float w3x = __shfl_sync(kAll, w.x, lead | 3), w3y = __shfl_sync(kAll, w.y, lead | 3),
                w3z = __shfl_sync(kAll, w.z, lead | 3);
    const float ax = k < 3 ? w.x - w3x : 0.f, ay = k < 3 ? w.y - w3y : 0.f, az = k < 3 ? w.z - w3z : 0.f;
    float H[3][3] = {{ax * b.x, ax * b.y, ax * b.z}, {ay * b.x, ay * b.y, ay * b.z}, {az * b.x, az * b.y, az * b.z}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            H[i][j] += __shfl_xor_sync(kAll, H[i][j], 1);
            H[i][j] += __shfl_xor_sync(kAll, H[i][j], 2);
        }
    const float V0 = __shfl_sync(kAll, b.w, lead);
    const float mu1 = __shfl_sync(kAll, mat.x, lead | 3), mu2 = __shfl_sync(kAll, mat.y, lead | 3),
                kappa = __shfl_sync(kAll, mat.z, lead | 3);
    InvT<float> v;
    float P[3][3];
    invariants_t(H, v);
    // FP64 J - 1 of a nearly incompressible tet: lane 0 gathers the columns
    // of A and broadcasts J - 1 (every lane takes part in the shuffles)
    float a1[3], a2[3];
    a1[0] = __shfl_sync(kAll, ax, lead | 1);
    a1[1] = __shfl_sync(kAll, ay, lead | 1);
    a1[2] = __shfl_sync(kAll, az, lead | 1);
    a2[0] = __shfl_sync(kAll, ax, lead | 2);
    a2[1] = __shfl_sync(kAll, ay, lead | 2);
    a2[2] = __shfl_sync(kAll, az, lead | 2);
    const bool fp64 = needs_fp64_volume(m, make_float4(mu1, mu2, kappa, 0.f));
    float j = v.j;
    if (fp64 && live && k == 0) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        j = (float)volume_change64_body(m.B64, m.T, t, make_float4(ax, ay, az, 0.f), make_float4(a1[0], a1[1], a1[2], 0.f),
                                        make_float4(a2[0], a2[1], a2[2], 0.f), z);
    }
    j = __shfl_sync(kAll, j, lead);
    if (fp64) set_volume_change(v, j);
    mr_stress_inv(H, mu1, mu2, kappa, v, P);
    if (live && k == 0 && !(v.J > 0.f)) atomicOr(err, ERR_INVERTED);
    float f[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) f[i] = k < 3 ? -V0 * (P[i][0] * b.x + P[i][1] * b.y + P[i][2] * b.z) : 0.f;
    float fs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        fs[i] = f[i] + __shfl_xor_sync(kAll, f[i], 1);
        fs[i] += __shfl_xor_sync(kAll, fs[i], 2);
    }
    if (k == 3) {
#pragma unroll
        for (int i = 0; i < 3; ++i) f[i] = -fs[i];
    }
    if (live) m.fc[(size_t)k * m.T + t] = make_float4(f[0], f[1], f[2], 0.f);
}

cudaError_t launch_tet_force(const MeshView &m, const float4 *u, unsigned *err, cudaStream_t s, int block,
                             int form, const LbmParams *lp, const RegionSlot *mark_out) {
    if (m.T == 0) return cudaSuccess;
    const int bs = block > 0 ? block : 64;  // default: ~20k tets still give every SM blocks
    const int cb = (lp && mark_out) ? (m.V + bs - 1) / bs : 0;
    const LbmParams p = lp ? *lp : LbmParams{};
    const RegionSlot mark = cb ? *mark_out : RegionSlot{nullptr};
    if (form == 2 && m.Bp) {
        const long long threads = 4LL * m.T;
        k_tet_force4<<<cb + (int)((threads + bs - 1) / bs), bs, 0, s>>>(m, u, err, cb, p, mark);
        return cudaGetLastError();
    }
    const int per = form == 1 ? 2 : 1;
    const int tb = (m.T + bs * per - 1) / (bs * per);
    if (per == 2)
        k_tet_force2<<<cb + tb, bs, 0, s>>>(m, u, err, cb, p, mark);
    else
        k_tet_force<<<cb + tb, bs, 0, s>>>(m, u, err, cb, p, mark);
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
        const int4 a4 = __ldg(m.tet + t);
        float Bm[3][3];
        load_B(m, t, Bm);
        float H[3][3];
        tet_grad(__ldg(u + a4.x), __ldg(u + a4.y), __ldg(u + a4.z), __ldg(u + a4.w), Bm, H);
        InvT<float> v;
        invariants_t(H, v);
        const float4 mat = __ldg(m.mat + mat_slot(m, t));
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
