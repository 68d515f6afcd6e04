// K1: Mooney-Rivlin nodal forces of every tet (Sec. 2, Sec. 3.1-3.2), one
// thread per tet, and the energy V_0 U per tet (K7, test support). The stress
// evaluation (the cancellation-free form of the paper's chain rule) is in
// mr.cuh.
#include "cell_ops.cuh"

namespace cf {

// The first mark_blocks blocks: one thread per vertex, marking the next
// step's force region. They come first so that their short, latency-bound
// work runs under the tets' rather than after it.
__device__ __forceinline__ void mark_block(const MeshView &m, const float4 *__restrict__ u, const LbmParams &lp,
                                           const RegionSlot &mark) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    if (lp.dw == 4)
        mark_vertex<4>(m, u, lp, v, mark);
    else
        mark_vertex<2>(m, u, lp, v, mark);
}

// Six blocks of 256 per SM (40 registers, a 16-byte spill): this latency-
// bound kernel gains more from the extra resident warps than the spill costs
// (tet forces of the 400-cell suspension 190.6 -> 178.5 us against 56
// registers and four blocks).
__global__ void __launch_bounds__(256, 6) k_tet_force(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                   int mark_blocks, LbmParams lp, RegionSlot mark) {
    if ((int)blockIdx.x < mark_blocks) {
        mark_block(m, u, lp, mark);
        return;
    }
    const int t = (blockIdx.x - mark_blocks) * blockDim.x + threadIdx.x;
    if (t >= m.T) return;

    tet_corner_forces(m, u, err, t);
}

// Two tets per thread, t and t + blockDim (coalesced either way): both tets'
// loads are issued before either is computed, doubling the bytes a thread
// has in flight in this latency-bound kernel.
__global__ void __launch_bounds__(256, 2) k_tet_force2(MeshView m, const float4 *__restrict__ u, unsigned *err,
                                                     int mark_blocks, LbmParams lp, RegionSlot mark) {
    if ((int)blockIdx.x < mark_blocks) {
        mark_block(m, u, lp, mark);
        return;
    }
    const int t0 = 2 * (blockIdx.x - mark_blocks) * blockDim.x + threadIdx.x, t1 = t0 + blockDim.x;
    if (t0 >= m.T) return;
    TetIn a, b;
    tet_load(m, u, t0, a);
    if (t1 < m.T) tet_load(m, u, t1, b);
    tet_forces_store(m, a, err, t0);
    if (t1 < m.T) tet_forces_store(m, b, err, t1);
}

cudaError_t launch_tet_force(const MeshView &m, const float4 *u, unsigned *err, cudaStream_t s, int block,
                             const LbmParams *lp, const RegionSlot *mark_out, int pairs) {
    if (m.T == 0) return cudaSuccess;
    const int bs = block > 0 ? block : 64;  // default: ~20k tets still give every SM blocks
    const int per = pairs ? 2 : 1;
    const int tb = (m.T + bs * per - 1) / (bs * per);
    const int cb = (lp && mark_out) ? (m.V + bs - 1) / bs : 0;
    const LbmParams p = lp ? *lp : LbmParams{};
    const RegionSlot mark = cb ? *mark_out : RegionSlot{nullptr, nullptr, nullptr};
    if (pairs)
        k_tet_force2<<<tb + cb, bs, 0, s>>>(m, u, err, cb, p, mark);
    else
        k_tet_force<<<tb + cb, bs, 0, s>>>(m, u, err, cb, p, mark);
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
