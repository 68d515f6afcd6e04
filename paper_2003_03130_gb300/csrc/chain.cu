// K1 + K23 as one persistent launch over all cells (the batched form of the
// cell chain): the per-vertex region marking (unless the interpolation of the
// step before marks the region), the tet corner forces (Sec. 3.1) and the
// vertex sums with their spread (Sec. 6), for cells of any size.
//
// Blocks take work items in a fixed order from one counter. Tet and region
// items never wait; a vertex-sum item of cell c waits until every tet item of
// cell c is done. The host orders the items so that every item an
// item waits for comes before it; the block holding an earlier item is
// therefore already running and never waits itself, so the waits end even
// when blocks are not co-resident or other kernels share the GPU. Each wait
// is still bounded: after spin_limit polls (a launch argument, by default
// 2^24 with a 64 ns back-off, about a second) it sets ERR_WAIT and the block
// skips the item. Vertex sums of early cells overlap the tet forces of later
// ones, and one launch replaces two.
#include "cell_ops.cuh"

namespace cf {

constexpr int kChainBlock = 256;

__device__ __forceinline__ int load_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_count(const int *p, int target, long long spin_limit, unsigned *err) {
    for (long long i = 0; i < spin_limit; ++i) {
        if (load_acquire(p) >= target) return true;
        __nanosleep(64);
    }
    atomicOr(err, ERR_WAIT);
    return false;
}

template <int W>
__global__ void __launch_bounds__(kChainBlock, 4)
    k_cell_chain(MeshView m, const float4 *__restrict__ u, float4 *F, LbmParams lp, RegionSlot mark, unsigned *err,
                 const int4 *__restrict__ items, int nitems, const int *__restrict__ need, int *counters,
                 long long spin_limit) {
    __shared__ int4 item;
    __shared__ int ready;
    int claim = 0;  // thread 0: the item claimed for the next round (claimed one round ahead)
    if (threadIdx.x == 0) claim = atomicAdd(counters, 1);
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = claim;
            const int4 x = i < nitems ? items[i] : make_int4(-1, 0, 0, 0);
            if (x.x >= 0) claim = atomicAdd(counters, 1);  // its latency hides under this item
            int ok = 1;
            if (x.x == 2) {
                ok = wait_count(counters + 2 + x.y, need[x.y], spin_limit, err);
                __threadfence();
            }
            item = x;
            ready = ok;
        }
        __syncthreads();
        const int4 x = item;
        if (x.x < 0) break;
        if (ready) {
            if (x.x == 0) {
                if (mark.bits)
                    for (int v = x.z + threadIdx.x; v < x.w; v += kChainBlock) mark_vertex<W>(m, u, lp, v, mark);
            } else if (x.x == 1) {
                for (int t = x.z + threadIdx.x; t < x.w; t += kChainBlock) tet_corner_forces(m, u, err, t);
            } else {
                for (int v0 = x.z; v0 < x.w; v0 += kChainBlock / 4) {  // the whole block takes each round
                    const int v = v0 + (threadIdx.x >> 2);
                    gather_spread_vertex<W, true>(m, u, F, lp, 1, err, v, threadIdx.x & 3, v < x.w);
                }
            }
        }
        __threadfence();  // this item's writes before its completion count
        __syncthreads();
        if (threadIdx.x == 0 && x.x == 1) atomicAdd(counters + 2 + x.y, 1);
    }
}

cudaError_t launch_cell_chain(const MeshView &m, const float4 *u, float4 *F, const LbmParams &lp,
                              const RegionSlot &mark, unsigned *err, const int4 *items, int nitems, const int *need,
                              int *counters, int blocks, long long spin_limit, cudaStream_t s) {
    if (nitems == 0) return cudaSuccess;
    const int g = blocks < nitems ? blocks : nitems;
    if (lp.dw == 4)
        k_cell_chain<4><<<g, kChainBlock, 0, s>>>(m, u, F, lp, mark, err, items, nitems, need, counters, spin_limit);
    else
        k_cell_chain<2><<<g, kChainBlock, 0, s>>>(m, u, F, lp, mark, err, items, nitems, need, counters, spin_limit);
    return cudaGetLastError();
}

}  // namespace cf
