// Immersed-boundary coupling (Sec. 6: the cell is coupled to the fluid by an
// immersed-boundary method; the kernel is not given there). Separable delta
// kernel of support width W per axis (internal.cuh): the trilinear two-point
// kernel (W = 2, 8 nodes per vertex) or Peskin's four-point kernel (W = 4,
// 64 nodes per vertex). Every vertex, interior ones included, is a coupling
// point (the fluid fills the cell).
//
// K2+K3 (k_gather_spread), four threads per vertex:
//   f_v = sum of the corner forces in the vertex's incidence row, in a fixed
//         order (strided partial sums combined by a fixed shuffle tree) -
//         deterministic, no atomics (Sec. 3.1 defines forces per tet corner;
//         the vertex force is their sum);
//   F(x) += f_v delta_h(x - y_v) on the W^3 support nodes: for W = 2 lane
//         (dz, dy) takes the two nodes of its x row, for W = 4 lane dz the
//         16 nodes of its z plane (float atomics: the spread field is exact
//         up to the order of those additions).
// K5 (k_interp_advect, eight threads per vertex, or k_interp_advect1, one):
//   y^{t+1} = y^t + sum_x u(x) delta_h(x - y^t), with u(t) as stored by the
//   near-field stream-collide on every node of the force region (which holds
//   the support of y^t), as eight partial sums of W^3 / 8 nodes each (for
//   W = 2 one corner (dz, dy, dx), for W = 4 the rows dy = 2j, 2j + 1 of a
//   plane dz) in a fixed tree, so both forms give the same bits. With
//   marking, the new position's support grown by one node is added to the
//   force region of step t + 2 (a vertex moves less than a spacing per step,
//   so that region holds the support of y^{t+2}).
#include <climits>

#include "cell_ops.cuh"

namespace cf {

// The force region of the current positions, into one or two slots (the
// first step of a call needs both its own region and the next step's, and
// the positions have not moved in between). Eight lanes per vertex share its
// tiles.
template <int W>
__global__ void __launch_bounds__(256) k_mark_region(MeshView m, const float4 *__restrict__ u, LbmParams p,
                                                     RegionSlot r, RegionSlot r2) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = g >> 3, lane = g & 7;
    Support s;
    if (v < m.V && support_of<W>(m.origin, __ldg(m.xr + v), __ldg(u + v), p.ny, s)) {
        mark_region<W>(s, p, r, lane, 8);
        if (r2.bits) mark_region<W>(s, p, r2, lane, 8);
    }
}

cudaError_t launch_mark_region(const MeshView &m, const float4 *u, const LbmParams &p, const RegionSlot &r,
                               const RegionSlot &r2, cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    const int blocks = (int)((8LL * m.V + 255) / 256);
    if (p.dw == 4)
        k_mark_region<4><<<blocks, 256, 0, s>>>(m, u, p, r, r2);
    else
        k_mark_region<2><<<blocks, 256, 0, s>>>(m, u, p, r, r2);
    return cudaGetLastError();
}

// K2+K3 with the spread staged in shared memory (launch shape: staged
// spread). A block takes 256 consecutive vertices (neighbours in the mesh's
// vertex order, so close in space), finds the bounding box of their delta
// supports, accumulates their spread into that box in shared memory (float
// atomics there), and adds each box node that received force to F with one
// float4 atomic. For the four-point kernel a vertex touches 64 nodes and a
// node receives about a dozen contributions, so the global atomics drop
// several-fold; for the trilinear kernel (8 nodes per vertex, ~2 per node)
// staging saves little. A box larger than kStageNodes (vertices of two
// cells, or a strongly stretched cell) falls back to global atomics for that
// block. The vertex sums are those of k_gather_spread (same order).
constexpr int kStageVerts = 256;
constexpr int kStageNodes = 6144;  // 3 x 24 KB of shared memory

template <int W>
__global__ void __launch_bounds__(256) k_gather_spread_staged(MeshView m, const float4 *__restrict__ u, float4 *F,
                                                              LbmParams p, unsigned *err) {
    extern __shared__ float stage[];  // [3][kStageNodes]: Fx, Fy, Fz of the box
    __shared__ int lo[3], hi[3];
    const int v0 = blockIdx.x * kStageVerts;
    if (threadIdx.x < 3) {
        lo[threadIdx.x] = INT_MAX;
        hi[threadIdx.x] = INT_MIN;
    }
    __syncthreads();
    {  // bounding box of the block's supports (lower corners; the box adds W - 1)
        const int v = v0 + threadIdx.x;
        Support s;
        if (v < m.V && support_of<W>(m.origin, __ldg(m.xr + v), __ldg(u + v), p.ny, s)) {
            atomicMin(lo + 0, s.bx);
            atomicMin(lo + 1, s.by);
            atomicMin(lo + 2, s.bz);
            atomicMax(hi + 0, s.bx);
            atomicMax(hi + 1, s.by);
            atomicMax(hi + 2, s.bz);
        }
    }
    __syncthreads();
    const int bx = hi[0] - lo[0] + W, by = hi[1] - lo[1] + W, bz = hi[2] - lo[2] + W;
    const bool staged = lo[0] != INT_MAX && (long long)bx * by * bz <= kStageNodes;
    const int vol = staged ? bx * by * bz : 0;
    for (int i = threadIdx.x; i < 3 * vol; i += blockDim.x) stage[(i / vol) * kStageNodes + i % vol] = 0.f;
    __syncthreads();
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int lane = threadIdx.x & 3;
    for (int k = threadIdx.x >> 2; k < kStageVerts; k += blockDim.x >> 2) {
        const int v = v0 + k;
        const bool live = v < m.V;
        float fx, fy, fz;
        gather_vertex<false>(m, v, lane, live, fx, fy, fz);
        if (!live) continue;
        if (lane == 0) {
            m.fv[v] = make_float4(fx, fy, fz, 0.f);
            if (!isfinite(fx + fy + fz)) atomicOr(err, ERR_NONFINITE);
        }
        Support s;
        if (!support_of<W>(m.origin, __ldg(m.xr + v), __ldg(u + v), p.ny, s)) {
            if (lane == 0) atomicOr(err, ERR_DOMAIN);
            continue;
        }
        if (staged) {
            spread_vertex<W>(s, lane, [&](int X, int Y, int Z, float w) {
                const int i = (X - lo[0]) + bx * ((Y - lo[1]) + by * (Z - lo[2]));
                atomicAdd(stage + i, w * fx);
                atomicAdd(stage + kStageNodes + i, w * fy);
                atomicAdd(stage + 2 * kStageNodes + i, w * fz);
            });
        } else {
            spread_vertex<W>(s, lane, [&](int X, int Y, int Z, float w) {
                const int n = wrapi(X, nx) + nx * (Y + ny * wrapi(Z, nz));
                force_add(F, p, n, w * fx, w * fy, w * fz);
            });
        }
    }
    if (!staged) return;
    __syncthreads();
    for (int i = threadIdx.x; i < vol; i += blockDim.x) {
        const float a = stage[i], b = stage[kStageNodes + i], c = stage[2 * kStageNodes + i];
        if (a == 0.f && b == 0.f && c == 0.f) continue;
        const int X = lo[0] + i % bx, Y = lo[1] + (i / bx) % by, Z = lo[2] + i / (bx * by);
        force_add(F, p, wrapi(X, nx) + nx * (Y + ny * wrapi(Z, nz)), a, b, c);
    }
}

template <int W>
__global__ void __launch_bounds__(256, 4) k_gather_spread(MeshView m, const float4 *__restrict__ u, float4 *F,
                                                          LbmParams p, int do_spread, unsigned *err) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = g >> 2;
    gather_spread_vertex<W, false>(m, u, F, p, do_spread, err, v, g & 3, v < m.V);
}

// The staged spread's box takes more than the default 48 KB of dynamic
// shared memory: opt in once per context, outside any stream capture.
cudaError_t prepare_staged_spread() {
    const int smem = (int)(3 * sizeof(float) * kStageNodes);
    cudaError_t e = cudaFuncSetAttribute(k_gather_spread_staged<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gather_spread_staged<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_gather_spread(const MeshView &m, const float4 *u, float4 *F, const LbmParams *lp, unsigned *err,
                                 cudaStream_t s, int block, int staged) {
    if (m.V == 0) return cudaSuccess;
    LbmParams p{};
    if (lp) p = *lp;
    if (staged && F && lp && !p.det) {  // shared-memory float sums would depend on their order
        const int blocks = (m.V + kStageVerts - 1) / kStageVerts;
        const size_t smem = 3 * sizeof(float) * kStageNodes;
        if (p.dw == 4)
            k_gather_spread_staged<4><<<blocks, 256, smem, s>>>(m, u, F, p, err);
        else
            k_gather_spread_staged<2><<<blocks, 256, smem, s>>>(m, u, F, p, err);
        return cudaGetLastError();
    }
    const int bs = block > 0 ? block : 128;
    const long long threads = 4LL * m.V;
    const int blocks = (int)((threads + bs - 1) / bs), spread = (F && lp) ? 1 : 0;
    if (p.dw == 4)
        k_gather_spread<4><<<blocks, bs, 0, s>>>(m, u, F, p, spread, err);
    else
        k_gather_spread<2><<<blocks, bs, 0, s>>>(m, u, F, p, spread, err);
    return cudaGetLastError();
}

// Eight threads per vertex, each one of the eight partial sums of the
// interpolation (interp_partial); the group of eight forms their tree by
// shuffles. MARK: the lanes also mark the region of the step after next (a
// separate instantiation, so that the form without marking keeps its lower
// register count).
template <int W, bool MARK>
__global__ void __launch_bounds__(256, 4) k_interp_advect(MeshView m, const float4 *__restrict__ vel, LbmParams p,
                                                       const float4 *__restrict__ u_cur, float4 *u_next,
                                                       unsigned *err, RegionSlot mark) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = g >> 3, lane = g & 7;
    const bool live = v < m.V;
    float4 uc = make_float4(0.f, 0.f, 0.f, 0.f), xr = uc;
    float3 a = make_float3(0.f, 0.f, 0.f);
    bool ok = false;
    if (live) {
        uc = __ldg(u_cur + v);
        xr = __ldg(m.xr + v);
        Support s;
        ok = support_of<W>(m.origin, xr, uc, p.ny, s);
        if (ok) {
            float wx[W], wy[W], wz[W];
            delta_weights<W>(s.fx, wx);
            delta_weights<W>(s.fy, wy);
            delta_weights<W>(s.fz, wz);
            a = interp_partial<W>(s, wx, wy, wz, vel, p, lane);
        }
    }
    // lane 0 ends with ((p0 + p1) + (p2 + p3)) + ((p4 + p5) + (p6 + p7))
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        a.x = __fadd_rn(a.x, __shfl_xor_sync(0xffffffffu, a.x, o));
        a.y = __fadd_rn(a.y, __shfl_xor_sync(0xffffffffu, a.y, o));
        a.z = __fadd_rn(a.z, __shfl_xor_sync(0xffffffffu, a.z, o));
    }
    if (!live) return;
    const float4 un = make_float4(__fadd_rn(uc.x, a.x), __fadd_rn(uc.y, a.y), __fadd_rn(uc.z, a.z), 0.f);
    if (MARK && ok) {  // the region of step t + 2 (an invalid support is K23's to report)
        Support s2;
        if (support_of<W>(m.origin, xr, un, p.ny, s2)) mark_region<W>(s2, p, mark, lane, 8);
    }
    if (lane != 0) return;
    if (!ok) {
        atomicOr(err, ERR_DOMAIN);
        u_next[v] = uc;
        return;
    }
    if (!isfinite(un.x + un.y + un.z)) atomicOr(err, ERR_NONFINITE);
    // the next step's force region holds this step's support grown by one
    // node: a move of a spacing or more along an axis would leave it
    if (!(fabsf(a.x) < 1.f && fabsf(a.y) < 1.f && fabsf(a.z) < 1.f)) atomicOr(err, ERR_MOVED);
    u_next[v] = un;
}

// One thread per vertex: the same partial sums and tree in one thread
// (fewer instructions per vertex than eight threads that each recompute the
// support and the weights; less parallelism for small meshes).
template <int W, bool MARK>
__global__ void __launch_bounds__(256) k_interp_advect1(MeshView m, const float4 *__restrict__ vel, LbmParams p,
                                                        const float4 *__restrict__ u_cur, float4 *u_next,
                                                        unsigned *err, RegionSlot mark) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const float4 uc = __ldg(u_cur + v), xr = __ldg(m.xr + v);
    Support s;
    float3 d;
    if (!interp_vertex<W>(m, vel, p, xr, uc, s, d)) {
        atomicOr(err, ERR_DOMAIN);
        u_next[v] = uc;
        return;
    }
    const float4 un = make_float4(__fadd_rn(uc.x, d.x), __fadd_rn(uc.y, d.y), __fadd_rn(uc.z, d.z), 0.f);
    if (MARK) {
        Support s2;
        if (support_of<W>(m.origin, xr, un, p.ny, s2)) mark_region<W>(s2, p, mark);
    }
    if (!isfinite(un.x + un.y + un.z)) atomicOr(err, ERR_NONFINITE);
    if (!(fabsf(d.x) < 1.f && fabsf(d.y) < 1.f && fabsf(d.z) < 1.f)) atomicOr(err, ERR_MOVED);
    u_next[v] = un;
}

template <int W, bool MARK>
static void interp_t(const MeshView &m, const float4 *vel, const LbmParams &p, const float4 *u_cur, float4 *u_next,
                     unsigned *err, cudaStream_t s, int bs, const RegionSlot &mark, int form) {
    if (form == 1) {
        k_interp_advect1<W, MARK><<<(m.V + bs - 1) / bs, bs, 0, s>>>(m, vel, p, u_cur, u_next, err, mark);
    } else {
        const long long threads = 8LL * m.V;
        k_interp_advect<W, MARK><<<(int)((threads + bs - 1) / bs), bs, 0, s>>>(m, vel, p, u_cur, u_next, err, mark);
    }
}

cudaError_t launch_interp_advect(const MeshView &m, const float4 *vel, const LbmParams &p, const float4 *u_cur,
                                 float4 *u_next, unsigned *err, cudaStream_t s, int block, const RegionSlot &mark,
                                 int form) {
    if (m.V == 0) return cudaSuccess;
    const int bs = block > 0 ? block : 128;
    const bool mk = mark.bits != nullptr;
    if (p.dw == 4) {
        if (mk)
            interp_t<4, true>(m, vel, p, u_cur, u_next, err, s, bs, mark, form);
        else
            interp_t<4, false>(m, vel, p, u_cur, u_next, err, s, bs, mark, form);
    } else {
        if (mk)
            interp_t<2, true>(m, vel, p, u_cur, u_next, err, s, bs, mark, form);
        else
            interp_t<2, false>(m, vel, p, u_cur, u_next, err, s, bs, mark, form);
    }
    return cudaGetLastError();
}

}  // namespace cf
