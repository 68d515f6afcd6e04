// Private to the library: the context behind the C ABI's opaque cf_ctx and
// the helpers shared by the translation units that implement the ABI.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cellfsi.h"
#include "internal.cuh"

namespace cf {

struct CellInfo {
    int v_off, nv, t_off, nt;
    int origin[3];
    float4 mat;
    bool per_tet = false;  // tets carry their own material slots (cf_set_tet_materials)
};

// Force-region tile shapes (log2 of the x, y, z extents; 256 nodes each).
constexpr int kTileShapes[4][3] = {{4, 2, 2}, {5, 2, 1}, {5, 1, 2}, {3, 3, 2}};
constexpr int kNumTileShapes = 4;

// Launch shapes of the step kernels. None changes a computed value: every
// kernel computes each tet, vertex or node the same way whatever its block.
struct Shape {
    int tile = 0;  // index into kTileShapes
    int tet_block = 64, gather_block = 128, interp_block = 128;
    int fused = 0;  // cell chain as one persistent launch (csrc/chain.cu) instead of two
    int near_rows = 0;  // near field in rows over the whole lattice instead of over the region's tile list
    int far_spec = 0;   // far field issues its loads before the region test resolves
    int tet_form = 0;   // force kernel: one thread per tet (0), two tets per thread (1), four lanes per tet (2)
    int pop_l2 = 0;     // FP32 far and near fields cache populations in L2 instead of streaming them
    int pop_pairs = 1;  // 16-bit formats, nx even: two nodes per thread in the row-form stream-collide
    int mark_k5 = 0;    // the interpolation (eight lanes per vertex) marks the region of the step after next,
                        // instead of the force launch (one thread per vertex) the next step's
    int staged = 0;     // the spread accumulates a block of vertices in shared memory before its global atomics
    int interp_form = 0;  // interpolation + advection: eight threads per vertex (0) or one (1)
};

}  // namespace cf

using namespace cf;

struct cf_ctx;
// Frees the compression/adjoint buffers and the tape (csrc/plates.cu).
void cf_free_adjoint(cf_ctx *c);

struct cf_ctx {
    using CellInfo = cf::CellInfo;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    double timeout_s = 600.0;

    // The device error word: kernels atomicOr ERR_* bits into d_err. Where the
    // device has native atomics on host memory, the word lives in mapped
    // page-locked memory (h_err, with d_err its device address) and the host
    // reads and clears it after a wait, with no copy on the stream; otherwise
    // d_err is device memory and h_err its page-locked copy.
    unsigned *d_err = nullptr;
    unsigned *h_err = nullptr;
    bool err_mapped = false;
    unsigned *seed = nullptr;  // rounding seeds of the two buffer parities (16-bit stochastic rounding)
    unsigned long long *d_status = nullptr;

    // fluid
    bool lbm_ready = false;
    LbmParams lp{};
    int pop_format = CF_POP_F32;  // CF_POP_* storage of the populations (next cf_lbm_init)
    int delta_w = 2;           // delta kernel support width (next cf_lbm_init)
    int spread_fixed = 0;      // deterministic (fixed-point) spread (next cf_lbm_init)
    void *f[2] = {nullptr, nullptr};
    float4 *F = nullptr;    // force field, (Fx, Fy, Fz, 0) per node, or fixed point long long [3][N]
    float4 *vel = nullptr;  // u(t) on the force region, (ux, uy, uz, 0) per node

    // cells
    int V = 0, T = 0;
    std::vector<CellInfo> cells;
    float4 *xr = nullptr, *u[2] = {nullptr, nullptr}, *fv = nullptr, *fc = nullptr;
    double *xref64 = nullptr;
    int4 *tet = nullptr;
    float *B = nullptr, *V0 = nullptr;
    double *B64 = nullptr;  // B in FP64 [9][T] (J - 1 of nearly incompressible tets)
    float4 *Bp = nullptr;  // packed B / V0 / cell rows for the force kernel, [3][T]
    int *tcell = nullptr, *origin = nullptr;
    int *tmat = nullptr;             // [T] material slot of each tet: its cell id, or a region slot
    std::vector<float4> rmats;       // region materials: slots ncells + i
    // work items of the fused cell chain (csrc/chain.cu), rebuilt when cells are added
    int4 *chain_items = nullptr;
    int *chain_need = nullptr, *chain_ctr = nullptr;
    int chain_nitems = 0;
    long long chain_spin_limit = 1LL << 24;  // polls before a wait of the fused chain gives up
    int chain_extra_need = 0;                // added to every cell's need count (cf_set_chain_wait)
    size_t mat_cap = 0;              // entries allocated in mat
    float4 *mat = nullptr;
    int *csr_ptr = nullptr, *csr_idx = nullptr, *csr_cursor = nullptr;
    double *energy_partial = nullptr, *energy_out = nullptr;
    double *stage = nullptr;  // [3 V] doubles for host <-> device vertex arrays
    double *taylor_partial = nullptr, *taylor_out = nullptr;

    // force regions: three slots of region_stride words, each the bitset over
    // the tiles of the current tiling (region_bits_max words for the tiling
    // with the most tiles)
    unsigned *region = nullptr;
    size_t region_stride = 0, region_bits_max = 0;
    // the tile form of the near field keeps running counts of the region
    // bitset in shared memory: false when they do not fit (lattices of more
    // than ~470 M nodes), and the near field then runs in rows
    bool near_tiles_fit = true;
    Shape shape;
    int sms = 152;  // multiprocessors of the device

    // compression between plates and its adjoint (csrc/plates.cu)
    struct TapeEntry {
        int n;
        float dt, c, kp;
        std::vector<float> zlo, zhi;
        int ck0, nck;  // checkpoints ck0 .. ck0 + nck - 1: steps 0, S, 2S, ..., and the end state
        std::vector<float4> mats;  // the cells' materials the call ran with
    };
    float k_plate = 0.f;
    std::vector<float> zlo_h, zhi_h;   // current plates per cell
    float *zlo = nullptr, *zhi = nullptr;
    std::vector<TapeEntry> tape;
    long long tape_gen = 0;            // bumped whenever the tape is emptied (cf_tape_clear, new cells)
    std::vector<float4 *> ckpt;        // device checkpoints: positions then velocities, 2 V float4 each
    int ck_used = 0;
    float4 *vel_r = nullptr;           // relaxation velocities [V]
    float4 *lam = nullptr, *lamv = nullptr, *mvec = nullptr, *jv = nullptr, *vtmp = nullptr;
    float4 *seg = nullptr, *segv = nullptr;  // positions / velocities of one segment, (stride + 1) x V
    double *grad = nullptr, *gtmp = nullptr, *pforce = nullptr, *dF = nullptr;
    int adj_V = 0, adj_C = 0;

    int cur = 0;          // buffer parity of the next step
    long long tstep = 0;  // steps taken; tstep % 3 picks the region slots
    int macro_tile = -1;  // tiling of the last step if it had cells (its region and u(t) there serve
                          // cf_get_velocity); -1: no such step since cf_lbm_init
    std::map<int, cudaGraphExec_t> graphs;
};

namespace {

cf_status fail(cf_ctx *c, cf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CUDA_TRY(c, expr)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail((c), e_ == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

template <class T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void drop_graphs(cf_ctx *c) {
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

MeshView view(const cf_ctx *c) {
    MeshView m;
    m.V = c->V;
    m.T = c->T;
    m.xr = c->xr;
    m.origin = c->origin;
    m.tet = c->tet;
    m.B = c->B;
    m.B64 = c->B64;
    m.Bp = c->Bp;
    m.V0 = c->V0;
    m.tcell = c->tcell;
    m.tmat = c->tmat;
    m.mat = c->mat;
    m.csr_ptr = c->csr_ptr;
    m.csr_idx = c->csr_idx;
    m.fc = c->fc;
    m.fv = c->fv;
    return m;
}

// Wait for the stream by polling, giving up after the context's timeout.
// The first 2 ms are spent polling (a step takes tens of microseconds, and a
// sleeping host thread would add its wake-up latency to every call); after
// that the thread sleeps 20 us between polls.
cf_status wait_stream(cf_ctx *c) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return CF_OK;
        if (e != cudaErrorNotReady) return fail(c, CF_ECUDA, "device work failed: %s", cudaGetErrorString(e));
        double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > c->timeout_s) return fail(c, CF_ETIMEOUT, "device work did not finish within %.0f s", c->timeout_s);
        if (dt > 2e-3) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Read and clear the device error word.
cf_status consume_errors(cf_ctx *c) {
    unsigned h = 0;
    if (c->err_mapped) {
        // every kernel of the context has finished after the wait, and the
        // word is written only by them
        cf_status s = wait_stream(c);
        if (s != CF_OK) return s;
        volatile unsigned *w = c->h_err;
        h = *w;
        *w = 0u;
    } else {
        // into page-locked memory the copy stays asynchronous, so the read
        // costs one wait instead of two
        CUDA_TRY(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
        cf_status s = wait_stream(c);
        if (s != CF_OK) return s;
        h = *c->h_err;
    }
    if (h & ERR_INVERTED) return fail(c, CF_EINVERTED, "a tet reached det F <= 0");
    if (h & ERR_NONFINITE) return fail(c, CF_ENONFINITE, "non-finite force or position");
    if (h & ERR_DOMAIN) return fail(c, CF_EDOMAIN, "a vertex's delta support left 0 <= y <= ny-1");
    if (h & ERR_MOVED) return fail(c, CF_EUNSTABLE, "a vertex moved a lattice spacing or more in one step");
    if (h & ERR_WAIT) return fail(c, CF_ETIMEOUT, "a bounded wait in the fused cell chain gave up");
    return CF_OK;
}

const CellInfo *cell_of(cf_ctx *c, int id) {
    if (!c || id < 0 || id >= (int)c->cells.size()) return nullptr;
    return &c->cells[id];
}

// Vertex range of a cell, or of all cells for CF_ALL_CELLS.
bool vertex_range(cf_ctx *c, int id, int *v0, int *nv) {
    if (!c) return false;
    if (id == CF_ALL_CELLS) {
        if (c->V == 0) return false;
        *v0 = 0;
        *nv = c->V;
        return true;
    }
    const CellInfo *ci = cell_of(c, id);
    if (!ci) return false;
    *v0 = ci->v_off;
    *nv = ci->nv;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now;
        cudaGetDevice(&now);
        if (prev >= 0 && now != prev) cudaSetDevice(prev);
    }
};

}  // namespace
