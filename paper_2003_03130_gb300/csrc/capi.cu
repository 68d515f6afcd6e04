// C ABI of libcellfsi.so (declared in include/cellfsi.h): context, device
// buffers, once-per-cell set-up and the coupled time step.
//
// One time step t -> t+1 (parity p) is, on the context's stream:
//   K1  tet forces at y^t (+ zero F on the support of y^{t-1})
//   K23 vertex sums over incidence rows + spread onto F
//   K4  stream + collide with F, populations f[p] -> f[1-p]
//   K5  interpolate u(t) at y^t, y^{t+1} = y^t + u  (u[p] -> u[1-p])
// With cells present, K4 is split by a force region around the cells: the
// far part (the tiles of 256 nodes outside the region, no force read) runs
// on a second stream concurrently with the cell chain
// K5(t-1) -> K1(t) -> K23(t); after the join the near part updates the
// region's tiles with the force field. The region of step t is the set of
// tiles that meet the delta support of y^{t-1} grown by one node (a vertex
// moves less than one spacing per step, so the support of y^t lies in it; K5
// checks every move and raises CF_EUNSTABLE otherwise). A cf_step call is a
// "first" step graph (region from the current positions, no K5 before it),
// n - 1 pipelined step graphs and a final K5; a one-step call is a single
// graph with its K5. Populations and displacements
// are double-buffered with one shared parity; each graph is captured once per
// parity. F keeps the last step's force until the next step begins, so the
// velocity of the last step can still be read.
#include <cuda_runtime.h>

#include <chrono>
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "ctx.h"

using namespace cf;

namespace {

// Steps per graph in the steady part of cf_step: even (buffer parity) and a
// multiple of 3 (region slots), so a graph starts and ends in the same phase.
constexpr int kChunk = 12;
// Calls of up to this many steps run as one graph (first step, the rest and
// the last K5); longer ones as the first step, chunks, one graph for the
// remainder and the last K5. Every graph boundary joins the two streams.
constexpr int kWhole = 24;

// First: the first step of a call (its region from the current positions);
// Mid: pipelined steps; Tail: K5 of the last step; Fluid: steps without
// cells; Single: a whole call of up to kWhole steps, the last K5 included
// (it waits for the near field only, so it overlaps the end of the far field).
enum class Kind { First = 0, Mid = 1, Tail = 2, Fluid = 3, Single = 4 };

// Region slots of step t (phase s = t % 3): the step's force region is slot
// (s + 2) % 3 (filled by step t - 1, or from the current positions in the
// first step of a call); the step fills the region of step t + 1 into slot
// s. Three slots keep a slot from being cleared while a far-field kernel two
// steps back may still read it.
size_t tiles_of(const LbmParams &p) { return (size_t)p.ntx * p.nty * p.ntz; }

RegionSlot slot_at(cf_ctx *c, int k) { return RegionSlot{c->region + c->region_stride * k}; }
RegionSlot region_slot(cf_ctx *c, int s) { return slot_at(c, (s + 2) % 3); }
RegionSlot accum_slot(cf_ctx *c, int s) { return slot_at(c, s); }

// Empty a slot: the bitset of the current tiling.
cudaError_t clear_slot(const cf_ctx *c, const RegionSlot &r, cudaStream_t s) {
    return cudaMemsetAsync(r.bits, 0, sizeof(unsigned) * ((tiles_of(c->lp) + 31) / 32), s);
}

int near_grid(const cf_ctx *c) { return 8 * c->sms; }
int chain_grid(const cf_ctx *c) { return 4 * c->sms; }

// Work items of the fused cell chain: the region items over all vertices
// (skipped by the kernel when the interpolation marks the region), then the
// tet items of the cells in order, with the vertex-sum items of a cell
// placed LAG items after its last tet item (by then its tets are most likely
// done, so the sums rarely wait), then the remaining vertex-sum items. Every
// item a vertex-sum item waits for comes before it.
cf_status build_chain_items(cf_ctx *c) {
    std::vector<int4> items;
    // item sizes: small meshes keep every block busy, large ones keep the
    // item count (one claim each) low
    const int grid = chain_grid(c);
    auto size_for = [&](int n, int lo, int hi) { return std::max(lo, std::min(hi, n / (2 * grid) / lo * lo)); };
    const int RB = size_for(c->V, 256, 1024), TB = size_for(c->T, 256, 1024), GB = size_for(c->V, 64, 256);
    const size_t LAG = 2 * (size_t)grid;
    for (int v = 0; v < c->V; v += RB) items.push_back(make_int4(0, 0, v, std::min(c->V, v + RB)));
    const int C = (int)c->cells.size();
    std::vector<int> need(C, 0);
    std::vector<size_t> last_tet(C, 0);
    auto gathers = [&](int k) {
        const CellInfo &ci = c->cells[k];
        for (int v = ci.v_off; v < ci.v_off + ci.nv; v += GB)
            items.push_back(make_int4(2, k, v, std::min(ci.v_off + ci.nv, v + GB)));
    };
    int next_sum = 0;  // first cell whose vertex sums are not placed yet
    for (int k = 0; k < C; ++k) {
        const CellInfo &ci = c->cells[k];
        for (int t = ci.t_off; t < ci.t_off + ci.nt; t += TB) {
            items.push_back(make_int4(1, k, t, std::min(ci.t_off + ci.nt, t + TB)));
            ++need[k];
            while (next_sum < k && items.size() >= last_tet[next_sum] + LAG) gathers(next_sum++);
        }
        last_tet[k] = items.size();
    }
    while (next_sum < C) gathers(next_sum++);
    for (int &n : need) n += c->chain_extra_need;
    dfree(c->chain_items);
    dfree(c->chain_need);
    dfree(c->chain_ctr);
    c->chain_nitems = 0;
    CUDA_TRY(c, dalloc(&c->chain_items, items.size()));
    CUDA_TRY(c, dalloc(&c->chain_need, std::max(C, 1)));
    CUDA_TRY(c, dalloc(&c->chain_ctr, 2 + std::max(C, 1)));
    CUDA_TRY(c, cudaMemcpyAsync(c->chain_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                c->stream));
    if (C) CUDA_TRY(c, cudaMemcpyAsync(c->chain_need, need.data(), sizeof(int) * C, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    c->chain_nitems = (int)items.size();
    return CF_OK;
}

// K1 + K23 of one step on stream s: the fused persistent launch, or the two
// separate kernels. Unless the interpolation marks the regions (mark_k5),
// K1 marks the next step's region into acc.
cudaError_t launch_chain_step(cf_ctx *c, const MeshView &m, int p, const Shape &sh, const RegionSlot &acc,
                              cudaStream_t s) {
    const RegionSlot none{nullptr};
    if (sh.fused) {
        cudaError_t e = cudaMemsetAsync(c->chain_ctr, 0, sizeof(int) * (2 + c->cells.size()), s);
        if (e != cudaSuccess) return e;
        return launch_cell_chain(m, c->u[p], c->F, c->lp, sh.mark_k5 ? none : acc, c->d_err, c->chain_items,
                                 c->chain_nitems, c->chain_need, c->chain_ctr, chain_grid(c), c->chain_spin_limit, s);
    }
    cudaError_t e = launch_tet_force(m, c->u[p], c->d_err, s, sh.tet_block, sh.tet_form, sh.mark_k5 ? nullptr : &c->lp,
                                     sh.mark_k5 ? nullptr : &acc);
    if (e != cudaSuccess) return e;
    return launch_gather_spread(m, c->u[p], c->F, &c->lp, c->d_err, s, sh.gather_block, sh.staged);
}

// Tile fields of the lattice parameters for tile shape k.
void set_tiles(LbmParams &p, int k) {
    p.tlx = kTileShapes[k][0];
    p.tly = kTileShapes[k][1];
    p.tlz = kTileShapes[k][2];
    p.ntx = (p.nx + (1 << p.tlx) - 1) >> p.tlx;
    p.nty = (p.ny + (1 << p.tly) - 1) >> p.tly;
    p.ntz = (p.nz + (1 << p.tlz) - 1) >> p.tlz;
}

// The lattice fields that follow the launch shape: tiles, L2 caching of
// FP32 populations, node pairs of the 16-bit formats.
void shape_to_lbm(LbmParams &p, const Shape &sh) {
    set_tiles(p, sh.tile);
    p.l2 = sh.pop_l2;
    p.pairs = sh.pop_pairs;
}

// Enqueue `nsteps` steps starting at parity p0 and phase s0 on two streams:
// sf carries the far-field stream-collide, sc the cell chain and the near
// field. ev holds 2 * nsteps + 1 events for the cross-stream dependencies:
//   far(t)   after far(t-1) [sf order] and near(t-1)
//   K5(t-1) -> K1(t) -> K23(t) after near(t-1) [sc order]
//   near(t)  after K23(t) [sc order] and far(t-1) (it reads far nodes' halo)
// so near(t) and the cell chain overlap far(t). The region of step t + 1
// (the support of y^t grown by one node) is marked by K1(t) or, with the
// launch shape's mark_k5, by K5(t-1), which computes y^t; the first step of
// a call marks its own region from the current positions (and, with
// mark_k5, the next one too).
cf_status enqueue_steps(cf_ctx *c, Kind kind, int p0, int s0, int nsteps, cudaStream_t sf, cudaStream_t sc,
                        cudaEvent_t *ev) {
    const MeshView m = view(c);
    const Shape &sh = c->shape;
    if (kind == Kind::Tail) {  // K5 of the last step (parity p0)
        CUDA_TRY(c, launch_interp_advect(m, c->vel, c->lp, c->u[p0], c->u[1 - p0], c->d_err, sf, sh.interp_block,
                                         RegionSlot{nullptr}, sh.interp_form));
        return CF_OK;
    }
    if (kind == Kind::Fluid) {
        for (int i = 0; i < nsteps; ++i) {
            const int p = p0 ^ (i & 1);
            CUDA_TRY(c, launch_lbm(c->f[p], c->f[1 - p], c->lp, c->seed + p, c->seed + 1 - p, sf));
        }
        return CF_OK;
    }
    cudaEvent_t fork = ev[0], *ev_far = ev + 1, *ev_near = ev + 1 + nsteps;
    const bool first = kind == Kind::First || kind == Kind::Single;
    const RegionSlot none{nullptr};
    if (first) {
        const RegionSlot use = region_slot(c, s0), acc = accum_slot(c, s0);
        CUDA_TRY(c, clear_slot(c, use, sf));
        if (sh.mark_k5) CUDA_TRY(c, clear_slot(c, acc, sf));
        CUDA_TRY(c, launch_mark_region(m, c->u[p0], c->lp, use, sh.mark_k5 ? acc : none, sf));
    }
    CUDA_TRY(c, cudaEventRecord(fork, sf));
    CUDA_TRY(c, cudaStreamWaitEvent(sc, fork, 0));
    for (int i = 0; i < nsteps; ++i) {
        const int p = p0 ^ (i & 1), s = (s0 + i) % 3;
        const RegionSlot use = region_slot(c, s), acc = accum_slot(c, s);
        if (i > 0) CUDA_TRY(c, cudaStreamWaitEvent(sf, ev_near[i - 1], 0));
        CUDA_TRY(c, launch_lbm_far(c->f[p], c->f[1 - p], c->lp, use.bits, c->seed + p, sh.far_spec, sf));
        CUDA_TRY(c, cudaEventRecord(ev_far[i], sf));
        if (!(first && i == 0)) {  // K5 of the previous step (parity 1-p), with mark_k5 marking acc
            if (sh.mark_k5) CUDA_TRY(c, clear_slot(c, acc, sc));
            CUDA_TRY(c, launch_interp_advect(m, c->vel, c->lp, c->u[1 - p], c->u[p], c->d_err, sc, sh.interp_block,
                                             sh.mark_k5 ? acc : none, sh.interp_form));
        }
        if (!sh.mark_k5) CUDA_TRY(c, clear_slot(c, acc, sc));
        CUDA_TRY(c, launch_chain_step(c, m, p, sh, acc, sc));
        if (i > 0) CUDA_TRY(c, cudaStreamWaitEvent(sc, ev_far[i - 1], 0));
        CUDA_TRY(c, launch_lbm_near(c->f[p], c->f[1 - p], c->F, c->lp, use.bits, c->vel,
                                    sh.near_rows || !c->near_tiles_fit ? 0 : near_grid(c), c->seed + p, c->seed + 1 - p, sc));
        CUDA_TRY(c, cudaEventRecord(ev_near[i], sc));
    }
    if (kind == Kind::Single) {  // K5 of the last step, after its near field in sc order
        const int pl = p0 ^ ((nsteps - 1) & 1);
        CUDA_TRY(c, launch_interp_advect(m, c->vel, c->lp, c->u[pl], c->u[1 - pl], c->d_err, sc, sh.interp_block,
                                         RegionSlot{nullptr}, sh.interp_form));
        CUDA_TRY(c, cudaEventRecord(ev_near[nsteps - 1], sc));
    }
    CUDA_TRY(c, cudaStreamWaitEvent(sf, ev_near[nsteps - 1], 0));
    CUDA_TRY(c, cudaStreamWaitEvent(sf, ev_far[nsteps - 1], 0));
    return CF_OK;
}

// Captured graph for (kind, parity, phase, steps), built on first use.
cf_status get_graph(cf_ctx *c, Kind kind, int p, int s, int nsteps, cudaGraphExec_t *out) {
    const int key = (((int)kind * 2 + p) * 3 + s) * 64 + nsteps;
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
        *out = it->second;
        return CF_OK;
    }
    // the cell chain runs at the highest stream priority so that its small
    // kernels get SMs as soon as far-field blocks retire
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    cudaStream_t sf = nullptr, sc = nullptr;
    std::vector<cudaEvent_t> ev(2 * nsteps + 1, nullptr);
    cf_status st = CF_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithPriority(&sf, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sc, cudaStreamNonBlocking, greatest);
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(sf, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = enqueue_steps(c, kind, p, s, nsteps, sf, sc, ev.data());
        e = cudaStreamEndCapture(sf, &g);
    }
    // every kernel node but the far field gets the highest priority
    if (e == cudaSuccess && st == CF_OK) {
        size_t nn = 0;
        e = cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
        for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
            cudaGraphNodeType ty;
            e = cudaGraphNodeGetType(nodes[i], &ty);
            if (e != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
            if (e != cudaSuccess) break;
            cudaLaunchAttributeValue v;
            v.priority = is_lbm_far_kernel(kp.func) ? least : greatest;
            e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaLaunchAttributePriority, &v);
        }
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && st == CF_OK) e = cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (sc) cudaStreamDestroy(sc);
    if (sf) cudaStreamDestroy(sf);
    if (st != CF_OK) return st;
    if (e != cudaSuccess) return fail(c, CF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    c->graphs[key] = exec;
    *out = exec;
    return CF_OK;
}

// Launch one graph of `nsteps` steps at the context's phase and advance it;
// with launch = false only make sure the graph exists.
cf_status launch_steps(cf_ctx *c, Kind kind, int nsteps, bool launch = true) {
    cudaGraphExec_t g;
    const int s = (int)(c->tstep % 3);
    cf_status st = get_graph(c, kind, c->cur, s, nsteps, &g);
    if (st != CF_OK) return st;
    if (launch) CUDA_TRY(c, cudaGraphLaunch(g, c->stream));
    c->cur ^= nsteps & 1;
    c->tstep += nsteps;
    return CF_OK;
}

// The graphs of n steps from the current state: with cells one graph for up
// to kWhole steps, else the first step, chunks of kChunk, the remainder,
// then K5 of the last step; or chunks of fluid-only steps and the remainder. launch = false instantiates them without running and
// leaves the state as it was.
cf_status schedule_steps(cf_ctx *c, int32_t n, bool launch) {
    const int cur0 = c->cur;
    const long long t0 = c->tstep;
    cf_status st = CF_OK;
    if (launch && n > 0) c->macro_tile = c->T > 0 ? c->shape.tile : -1;
    if (c->T == 0) {
        int left = n;
        while (st == CF_OK && left >= kChunk) {
            st = launch_steps(c, Kind::Fluid, kChunk, launch);
            left -= kChunk;
        }
        if (st == CF_OK && left > 0) st = launch_steps(c, Kind::Fluid, left, launch);
    } else {
        if (n <= kWhole) {  // one graph for the whole call
            st = launch_steps(c, Kind::Single, n, launch);
            if (!launch) {
                c->cur = cur0;
                c->tstep = t0;
            }
            return st;
        }
        st = launch_steps(c, Kind::First, 1, launch);
        int left = n - 1;
        while (st == CF_OK && left >= kChunk) {
            st = launch_steps(c, Kind::Mid, kChunk, launch);
            left -= kChunk;
        }
        if (st == CF_OK && left > 0) st = launch_steps(c, Kind::Mid, left, launch);
        cudaGraphExec_t g;
        if (st == CF_OK) st = get_graph(c, Kind::Tail, c->cur ^ 1, 0, 1, &g);  // parity of the last step
        if (st == CF_OK && launch) CUDA_TRY(c, cudaGraphLaunch(g, c->stream));
    }
    if (!launch) {
        c->cur = cur0;
        c->tstep = t0;
    }
    return st;
}

}  // namespace

extern "C" {

cf_status cf_create(cf_ctx **out, int device, void *cuda_stream) {
    if (!out) return CF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return CF_EINVAL;
    cf_ctx *c = new cf_ctx();
    c->device = device;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->sms < 1)
        c->sms = 152;
    if (const char *t = getenv("CELLFSI_TIMEOUT_S")) c->timeout_s = atof(t);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return CF_ECUDA;
        }
        c->own_stream = true;
    }
    int host_atomics = 0;
    if (cudaDeviceGetAttribute(&host_atomics, cudaDevAttrHostNativeAtomicSupported, device) != cudaSuccess)
        host_atomics = 0;
    if (host_atomics && cudaHostAlloc((void **)&c->h_err, sizeof(unsigned), cudaHostAllocMapped) == cudaSuccess) {
        *c->h_err = 0u;
        if (cudaHostGetDevicePointer((void **)&c->d_err, c->h_err, 0) == cudaSuccess) {
            c->err_mapped = true;
        } else {
            cudaGetLastError();
            cudaFreeHost(c->h_err);
            c->h_err = nullptr;
            c->d_err = nullptr;
        }
    } else {
        cudaGetLastError();
        c->h_err = nullptr;
    }
    const bool err_ok =
        c->err_mapped || (dalloc(&c->d_err, 1) == cudaSuccess && cudaMemset(c->d_err, 0, sizeof(unsigned)) == cudaSuccess &&
                          cudaMallocHost((void **)&c->h_err, sizeof(unsigned)) == cudaSuccess);
    if (!err_ok || dalloc(&c->d_status, 1) != cudaSuccess || dalloc(&c->taylor_out, 10) != cudaSuccess ||
        dalloc(&c->seed, 2) != cudaSuccess || cudaMemset(c->seed, 0, 2 * sizeof(unsigned)) != cudaSuccess ||
        dalloc(&c->energy_out, 1) != cudaSuccess) {
        cf_destroy(c);
        return CF_ENOMEM;
    }
    if (prepare_staged_spread() != cudaSuccess) {
        cf_destroy(c);
        return CF_ECUDA;
    }
    *out = c;
    return CF_OK;
}

void cf_destroy(cf_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (!c->err_mapped) dfree(c->d_err);  // else the device address of h_err
    dfree(c->d_status);
    dfree(c->seed);
    if (c->h_err) cudaFreeHost(c->h_err);
    dfree(c->region);
    dfree(c->f[0]);
    dfree(c->f[1]);
    dfree(c->F);
    dfree(c->vel);
    dfree(c->xr);
    dfree(c->u[0]);
    dfree(c->u[1]);
    dfree(c->fv);
    dfree(c->fc);
    dfree(c->xref64);
    dfree(c->tet);
    dfree(c->B);
    dfree(c->B64);
    dfree(c->Bp);
    dfree(c->V0);
    dfree(c->tcell);
    dfree(c->tmat);
    dfree(c->chain_items);
    dfree(c->chain_need);
    dfree(c->chain_ctr);
    dfree(c->origin);
    dfree(c->mat);
    dfree(c->csr_ptr);
    dfree(c->csr_idx);
    dfree(c->csr_cursor);
    dfree(c->energy_partial);
    dfree(c->energy_out);
    dfree(c->stage);
    dfree(c->taylor_partial);
    dfree(c->taylor_out);
    cf_free_adjoint(c);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *cf_last_error(const cf_ctx *c) { return c ? c->err.c_str() : "null context"; }

cf_status cf_lbm_init(cf_ctx *c, int32_t nx, int32_t ny, int32_t nz, double tau, double u_lo, double u_hi,
                      const double *g) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (nx < 1 || ny < 1 || nz < 1) return fail(c, CF_EINVAL, "lattice extents must be >= 1");
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 30)) return fail(c, CF_EINVAL, "lattice too large: nx*ny*nz must be < 2^30");
    if (ny > 65535 || nz > 65535) return fail(c, CF_EINVAL, "ny and nz must be <= 65535 (rows are grid dimensions)");
    if (!(tau > 0.5)) return fail(c, CF_EINVAL, "tau must be > 1/2");
    if (!(std::fabs(u_lo) < 0.1 && std::fabs(u_hi) < 0.1)) return fail(c, CF_EINVAL, "|u_wall| must be < 0.1");
    if (g && !(std::isfinite(g[0]) && std::isfinite(g[1]) && std::isfinite(g[2])))
        return fail(c, CF_EINVAL, "body force must be finite");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    dfree(c->f[0]);
    dfree(c->f[1]);
    dfree(c->F);
    dfree(c->vel);
    dfree(c->region);
    c->lbm_ready = false;
    LbmParams p{};
    p.fmt = c->pop_format == CF_POP_F16_SR ? POP_F16 : c->pop_format == CF_POP_BF16_SR ? POP_BF16 : c->pop_format;
    p.sr = c->pop_format == CF_POP_F16_SR || c->pop_format == CF_POP_BF16_SR;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = N;
    p.omega = (float)(1.0 / tau);
    p.guo = (float)(1.0 - 0.5 / tau);
    p.uw_lo = (float)u_lo;
    p.uw_hi = (float)u_hi;
    p.gx = g ? (float)g[0] : 0.f;
    p.gy = g ? (float)g[1] : 0.f;
    p.gz = g ? (float)g[2] : 0.f;
    p.dw = c->delta_w;
    p.det = c->spread_fixed;
    // region slots sized for the largest tile count of any tile shape
    size_t tmax = 0;
    for (int k = 0; k < kNumTileShapes; ++k) {
        set_tiles(p, k);
        tmax = std::max(tmax, tiles_of(p));
    }
    shape_to_lbm(p, c->shape);
    c->region_bits_max = (tmax + 31) / 32;
    c->region_stride = (c->region_bits_max + 31) / 32 * 32;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    c->near_tiles_fit = sizeof(int) * (c->region_bits_max + 1) + 256 <= (size_t)smem_optin;  // + static
    if (c->near_tiles_fit && prepare_near_field((long long)c->region_bits_max) != cudaSuccess)
        return fail(c, CF_ECUDA, "shared-memory opt-in of the near field failed");
    const size_t pop = pop_bytes(p.fmt) * 19 * (size_t)N;
    CUDA_TRY(c, cudaMalloc(&c->f[0], pop));
    CUDA_TRY(c, cudaMalloc(&c->f[1], pop));
    // float4 per node, or long long [3][N] for the deterministic spread
    const size_t f_units = p.det ? (3 * (size_t)N + 1) / 2 : (size_t)N;
    CUDA_TRY(c, dalloc(&c->F, f_units));
    CUDA_TRY(c, dalloc(&c->vel, (size_t)N));
    CUDA_TRY(c, dalloc(&c->region, 3 * c->region_stride));
    CUDA_TRY(c, cudaMemsetAsync(c->region, 0, sizeof(unsigned) * 3 * c->region_stride, c->stream));
    CUDA_TRY(c, launch_lbm_init(c->f[0], p, c->stream));
    CUDA_TRY(c, launch_lbm_init(c->f[1], p, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->F, 0, sizeof(float4) * f_units, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->vel, 0, sizeof(float4) * (size_t)N, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->seed, 0, 2 * sizeof(unsigned), c->stream));  // rounding seeds restart
    c->lp = p;
    c->macro_tile = -1;
    c->lbm_ready = true;
    return wait_stream(c);
}

cf_status cf_set_population_format(cf_ctx *c, int32_t format) {
    if (!c) return CF_EINVAL;
    if (format != CF_POP_F32 && format != CF_POP_F16 && format != CF_POP_BF16 && format != CF_POP_F16_SR &&
        format != CF_POP_BF16_SR)
        return fail(c, CF_EINVAL, "unknown population format %d", format);
    c->pop_format = format;
    return CF_OK;
}

cf_status cf_set_spread(cf_ctx *c, int32_t mode) {
    if (!c) return CF_EINVAL;
    if (mode != CF_SPREAD_FLOAT && mode != CF_SPREAD_FIXED) return fail(c, CF_EINVAL, "unknown spread mode %d", mode);
    c->spread_fixed = mode == CF_SPREAD_FIXED;
    return CF_OK;
}

cf_status cf_set_delta(cf_ctx *c, int32_t kernel) {
    if (!c) return CF_EINVAL;
    if (kernel != CF_DELTA_TRILINEAR && kernel != CF_DELTA_PESKIN4)
        return fail(c, CF_EINVAL, "unknown delta kernel %d", kernel);
    c->delta_w = kernel;
    return CF_OK;
}

cf_status cf_mesh_init_batch(cf_ctx *c, int32_t ncells, const int32_t *nv, const double *x_ref, const int32_t *nt,
                             const int32_t *tets, const double *y0, int32_t *cell_ids_out) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (ncells < 1 || !nv || !nt || !x_ref || !tets) return fail(c, CF_EINVAL, "need ncells >= 1 and non-null arrays");
    // per-cell offsets into the concatenated inputs, origins, validation
    std::vector<long long> voff(ncells + 1, 0), toff(ncells + 1, 0);
    std::vector<CellInfo> add(ncells);
    for (int k = 0; k < ncells; ++k) {
        if (nv[k] < 4 || nt[k] < 1) return fail(c, CF_EINVAL, "cell %d: need nv >= 4 and nt >= 1", k);
        voff[k + 1] = voff[k] + nv[k];
        toff[k + 1] = toff[k] + nt[k];
    }
    if (c->T + toff[ncells] > INT_MAX / 4 || c->V + voff[ncells] > INT_MAX / 4)
        return fail(c, CF_EINVAL, "mesh too large");
    for (int k = 0; k < ncells; ++k) {
        double mean[3] = {0, 0, 0};
        for (long long v = voff[k]; v < voff[k + 1]; ++v)
            for (int a = 0; a < 3; ++a) {
                if (!std::isfinite(x_ref[3 * v + a]) || (y0 && !std::isfinite(y0[3 * v + a])))
                    return fail(c, CF_EINVAL, "cell %d: non-finite coordinate at vertex %lld", k, v - voff[k]);
                mean[a] += x_ref[3 * v + a];
            }
        CellInfo &ci = add[k];
        ci.v_off = c->V + (int)voff[k];
        ci.nv = nv[k];
        ci.t_off = c->T + (int)toff[k];
        ci.nt = nt[k];
        for (int a = 0; a < 3; ++a) ci.origin[a] = (int)std::lround(mean[a] / nv[k]);
        ci.mat = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int Vadd = (int)voff[ncells], Tadd = (int)toff[ncells];
    const int V1 = c->V + Vadd, T1 = c->T + Tadd, cell0 = (int)c->cells.size(), C1 = cell0 + ncells;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));

    // new arrays; the old ones are freed only on success
    cf_ctx n;  // holder for the new buffers (never destroyed as a context)
    double *x64 = nullptr, *y64 = nullptr;
    int *tin = nullptr;
    auto cleanup = [&]() {
        dfree(n.xr); dfree(n.u[0]); dfree(n.u[1]); dfree(n.fv); dfree(n.fc); dfree(n.xref64); dfree(n.tet);
        dfree(n.B); dfree(n.B64); dfree(n.Bp); dfree(n.V0); dfree(n.tcell); dfree(n.tmat); dfree(n.origin); dfree(n.mat); dfree(n.csr_ptr);
        dfree(n.csr_idx); dfree(n.csr_cursor); dfree(n.energy_partial); dfree(n.stage); dfree(n.taylor_partial);
        dfree(x64); dfree(y64); dfree(tin);
    };
#define TRY_N(expr)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            cleanup();                                                                                 \
            return fail(c, e_ == cudaErrorMemoryAllocation ? CF_ENOMEM : CF_ECUDA, "%s: %s", #expr,   \
                        cudaGetErrorString(e_));                                                       \
        }                                                                                              \
    } while (0)
    TRY_N(dalloc(&n.xr, V1));
    TRY_N(dalloc(&n.u[0], V1));
    TRY_N(dalloc(&n.u[1], V1));
    TRY_N(dalloc(&n.fv, V1));
    TRY_N(dalloc(&n.fc, 4 * (size_t)T1));
    TRY_N(dalloc(&n.xref64, 3 * (size_t)V1));
    TRY_N(dalloc(&n.tet, T1));
    TRY_N(dalloc(&n.B, 9 * (size_t)T1));
    TRY_N(dalloc(&n.B64, 9 * (size_t)T1));
    TRY_N(dalloc(&n.Bp, 3 * (size_t)T1));
    TRY_N(dalloc(&n.V0, T1));
    TRY_N(dalloc(&n.tcell, T1));
    TRY_N(dalloc(&n.tmat, T1));
    TRY_N(dalloc(&n.origin, 3 * (size_t)C1));
    TRY_N(dalloc(&n.mat, C1 + c->rmats.size()));
    TRY_N(dalloc(&n.csr_ptr, V1 + 1));
    TRY_N(dalloc(&n.csr_idx, 4 * (size_t)T1));
    TRY_N(dalloc(&n.csr_cursor, V1));
    TRY_N(dalloc(&n.energy_partial, (T1 + 255) / 256 + 1));
    TRY_N(dalloc(&n.stage, 3 * (size_t)V1));
    TRY_N(dalloc(&n.taylor_partial, 10 * ((size_t)(T1 + 255) / 256 + 1)));
    TRY_N(dalloc(&x64, 3 * (size_t)Vadd));
    TRY_N(dalloc(&tin, 4 * (size_t)Tadd));
    if (y0) TRY_N(dalloc(&y64, 3 * (size_t)Vadd));
    cudaStream_t s = c->stream;
    if (c->V > 0) {
        TRY_N(cudaMemcpyAsync(n.xr, c->xr, sizeof(float4) * c->V, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.u[0], c->u[0], sizeof(float4) * c->V, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.u[1], c->u[1], sizeof(float4) * c->V, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.xref64, c->xref64, sizeof(double) * 3 * c->V, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.tet, c->tet, sizeof(int4) * c->T, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpy2DAsync(n.B, sizeof(float) * T1, c->B, sizeof(float) * c->T, sizeof(float) * c->T, 9,
                                cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpy2DAsync(n.B64, sizeof(double) * T1, c->B64, sizeof(double) * c->T, sizeof(double) * c->T, 9,
                                cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.V0, c->V0, sizeof(float) * c->T, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.tcell, c->tcell, sizeof(int) * c->T, cudaMemcpyDeviceToDevice, s));
        TRY_N(cudaMemcpyAsync(n.tmat, c->tmat, sizeof(int) * c->T, cudaMemcpyDeviceToDevice, s));
        TRY_N(launch_shift_slots(c->T, cell0, ncells, n.tmat, s));  // region slots follow the cells
    }
    std::vector<int> orig(3 * (size_t)C1);
    std::vector<float4> mats(C1 + c->rmats.size());
    for (int i = 0; i < cell0; ++i) {
        for (int a = 0; a < 3; ++a) orig[3 * i + a] = c->cells[i].origin[a];
        mats[i] = c->cells[i].mat;
    }
    for (int k = 0; k < ncells; ++k) {
        for (int a = 0; a < 3; ++a) orig[3 * (cell0 + k) + a] = add[k].origin[a];
        mats[cell0 + k] = add[k].mat;
    }
    for (size_t i = 0; i < c->rmats.size(); ++i) mats[C1 + i] = c->rmats[i];
    TRY_N(cudaMemcpyAsync(n.origin, orig.data(), sizeof(int) * orig.size(), cudaMemcpyHostToDevice, s));
    TRY_N(cudaMemcpyAsync(n.mat, mats.data(), sizeof(float4) * mats.size(), cudaMemcpyHostToDevice, s));
    TRY_N(cudaMemcpyAsync(x64, x_ref, sizeof(double) * 3 * Vadd, cudaMemcpyHostToDevice, s));
    TRY_N(cudaMemcpyAsync(tin, tets, sizeof(int) * 4 * (size_t)Tadd, cudaMemcpyHostToDevice, s));
    if (y0) TRY_N(cudaMemcpyAsync(y64, y0, sizeof(double) * 3 * Vadd, cudaMemcpyHostToDevice, s));
    TRY_N(cudaMemsetAsync(c->d_status, 0xff, sizeof(unsigned long long), s));
    for (int k = 0; k < ncells; ++k)
        TRY_N(launch_mesh_prepare(x64 + 3 * voff[k], nv[k], tin + 4 * toff[k], nt[k], add[k].v_off, add[k].t_off,
                                  (int)toff[k], T1, cell0 + k, n.tet, n.B, n.B64, n.V0, n.tcell, c->d_status, s));
    unsigned long long st = 0;
    TRY_N(cudaMemcpyAsync(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost, s));
    TRY_N(cudaStreamSynchronize(s));
    if (st != ~0ULL) {
        cleanup();
        const int code = (int)(st & 0xff);
        const long long bad = (long long)(st >> 8);  // tet index within the batch
        int k = 0;
        while (k + 1 < ncells && toff[k + 1] <= bad) ++k;
        const int local = (int)(bad - toff[k]);
        if (code == 3) return fail(c, CF_EDEGENERATE, "cell %d, tet %d is degenerate (|det J| <= 1e-12 l^3)", k, local);
        return fail(c, CF_EINVAL, "cell %d, tet %d: %s", k, local,
                    code == 1 ? "vertex index out of range" : "repeated vertex");
    }
    for (int k = 0; k < ncells; ++k)
        TRY_N(launch_vertex_prepare(x64 + 3 * voff[k], y64 ? y64 + 3 * voff[k] : nullptr, nv[k], add[k].v_off,
                                    cell0 + k, add[k].origin, n.xr, n.u[0], n.u[1], n.xref64, s));
    TRY_N(launch_csr_build(n.tet, T1, V1, n.csr_ptr, n.csr_idx, n.csr_cursor, s));
    TRY_N(cudaMemcpyAsync(n.tmat + c->T, n.tcell + c->T, sizeof(int) * (T1 - c->T), cudaMemcpyDeviceToDevice, s));
    TRY_N(launch_pack_tets(T1, n.B, n.V0, n.tmat, n.Bp, s));
    TRY_N(cudaStreamSynchronize(s));
#undef TRY_N
    dfree(x64);
    dfree(y64);
    dfree(tin);
    drop_graphs(c);
    std::swap(c->xr, n.xr);
    std::swap(c->u[0], n.u[0]);
    std::swap(c->u[1], n.u[1]);
    std::swap(c->fv, n.fv);
    std::swap(c->fc, n.fc);
    std::swap(c->xref64, n.xref64);
    std::swap(c->tet, n.tet);
    std::swap(c->B, n.B);
    std::swap(c->B64, n.B64);
    std::swap(c->Bp, n.Bp);
    std::swap(c->V0, n.V0);
    std::swap(c->tcell, n.tcell);
    std::swap(c->tmat, n.tmat);
    std::swap(c->origin, n.origin);
    std::swap(c->mat, n.mat);
    c->mat_cap = C1 + c->rmats.size();
    std::swap(c->csr_ptr, n.csr_ptr);
    std::swap(c->csr_idx, n.csr_idx);
    std::swap(c->csr_cursor, n.csr_cursor);
    std::swap(c->energy_partial, n.energy_partial);
    std::swap(c->stage, n.stage);
    std::swap(c->taylor_partial, n.taylor_partial);
    cleanup();  // frees the old buffers now held by n
    c->V = V1;
    c->T = T1;
    for (int k = 0; k < ncells; ++k) {
        c->cells.push_back(add[k]);
        if (cell_ids_out) cell_ids_out[k] = cell0 + k;
    }
    return build_chain_items(c);
}

cf_status cf_mesh_init(cf_ctx *c, int32_t nv, const double *x_ref, int32_t nt, const int32_t *tets, const double *y0,
                       int32_t *cell_id_out) {
    return cf_mesh_init_batch(c, 1, &nv, x_ref, &nt, tets, y0, cell_id_out);
}

}  // extern "C"

namespace {

bool material_ok(double mu, double kappa, double w) {
    return mu >= 0.0 && kappa >= 0.0 && w >= 0.0 && w <= 1.0 && std::isfinite(mu) && std::isfinite(kappa);
}

float4 material_of(double mu, double kappa, double w) {
    return make_float4((float)(w * mu), (float)((1.0 - w) * mu), (float)kappa, (float)w);
}

// Upload the material table [cells..., region slots...] (grown when needed).
cf_status upload_materials(cf_ctx *c) {
    std::vector<float4> mats(c->cells.size() + c->rmats.size());
    for (size_t i = 0; i < c->cells.size(); ++i) mats[i] = c->cells[i].mat;
    for (size_t i = 0; i < c->rmats.size(); ++i) mats[c->cells.size() + i] = c->rmats[i];
    if (mats.empty()) return CF_OK;
    if (mats.size() > c->mat_cap) {
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // no kernel still reads the old table
        float4 *grown = nullptr;
        CUDA_TRY(c, dalloc(&grown, mats.size()));
        dfree(c->mat);
        c->mat = grown;
        c->mat_cap = mats.size();
        drop_graphs(c);  // captured launches hold the old table's address
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->mat, mats.data(), sizeof(float4) * mats.size(), cudaMemcpyHostToDevice,
                                c->stream));
    return CF_OK;
}

// Point the tets of a cell at material slots (slot ids on the host, or the
// cell's own slot when null) and refresh the packed rows.
cf_status set_tet_slots(cf_ctx *c, int id, const int *slots) {
    const CellInfo &ci = c->cells[id];
    if (slots) {
        CUDA_TRY(c, cudaMemcpyAsync(c->tmat + ci.t_off, slots, sizeof(int) * ci.nt, cudaMemcpyHostToDevice,
                                    c->stream));
    } else {
        CUDA_TRY(c, cudaMemcpyAsync(c->tmat + ci.t_off, c->tcell + ci.t_off, sizeof(int) * ci.nt,
                                    cudaMemcpyDeviceToDevice, c->stream));
    }
    CUDA_TRY(c, launch_pack_tets(c->T, c->B, c->V0, c->tmat, c->Bp, c->stream));
    return CF_OK;
}

}  // namespace

extern "C" {

cf_status cf_set_materials(cf_ctx *c, int32_t ncells, const int32_t *ids, const double *mu, const double *kappa,
                           const double *w) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (ncells < 0 || (ncells > 0 && (!ids || !mu || !kappa || !w))) return fail(c, CF_EINVAL, "null arrays");
    for (int k = 0; k < ncells; ++k) {
        if (ids[k] < 0 || ids[k] >= (int)c->cells.size()) return fail(c, CF_EINVAL, "unknown cell %d", ids[k]);
        if (!material_ok(mu[k], kappa[k], w[k]))
            return fail(c, CF_EINVAL, "cell %d: need mu >= 0, kappa >= 0, 0 <= w <= 1", ids[k]);
    }
    for (int k = 0; k < ncells; ++k) {
        CellInfo &ci = c->cells[ids[k]];
        ci.mat = material_of(mu[k], kappa[k], w[k]);
        if (ci.per_tet) {  // uniform again
            cf_status st = set_tet_slots(c, ids[k], nullptr);
            if (st != CF_OK) return st;
            ci.per_tet = false;
        }
    }
    cf_status st = upload_materials(c);
    return st != CF_OK ? st : wait_stream(c);
}

cf_status cf_set_material(cf_ctx *c, int32_t id, double mu, double kappa, double w) {
    return cf_set_materials(c, 1, &id, &mu, &kappa, &w);
}

cf_status cf_set_tet_materials(cf_ctx *c, int32_t id, const int32_t *region, int32_t nreg, const double *mu,
                               const double *kappa, const double *w) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (id < 0 || id >= (int)c->cells.size()) return fail(c, CF_EINVAL, "unknown cell %d", id);
    if (nreg < 1 || !region || !mu || !kappa || !w) return fail(c, CF_EINVAL, "need nreg >= 1 and non-null arrays");
    for (int r = 0; r < nreg; ++r)
        if (!material_ok(mu[r], kappa[r], w[r]))
            return fail(c, CF_EINVAL, "region %d: need mu >= 0, kappa >= 0, 0 <= w <= 1", r);
    CellInfo &ci = c->cells[id];
    const int base = (int)(c->cells.size() + c->rmats.size());
    std::vector<int> slots(ci.nt);
    for (int t = 0; t < ci.nt; ++t) {
        if (region[t] < 0 || region[t] >= nreg)
            return fail(c, CF_EINVAL, "tet %d: region %d out of [0, %d)", t, region[t], nreg);
        slots[t] = base + region[t];
    }
    for (int r = 0; r < nreg; ++r) c->rmats.push_back(material_of(mu[r], kappa[r], w[r]));
    cf_status st = upload_materials(c);
    if (st == CF_OK) st = set_tet_slots(c, id, slots.data());
    if (st == CF_OK) ci.per_tet = true;
    return st != CF_OK ? st : wait_stream(c);
}

cf_status cf_step_async(cf_ctx *c, int32_t n) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (n < 0) return fail(c, CF_EINVAL, "n must be >= 0");
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "cf_step needs cf_lbm_init first");
    if (n == 0) return CF_OK;
    return schedule_steps(c, n, true);
}

cf_status cf_prepare_steps(cf_ctx *c, int32_t n) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (n < 0) return fail(c, CF_EINVAL, "n must be >= 0");
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "cf_prepare_steps needs cf_lbm_init first");
    if (n == 0) return CF_OK;
    // the graphs depend on the buffer parity and the region phase: build them
    // for all six states, then put the state back
    const int cur0 = c->cur;
    const long long t0 = c->tstep;
    cf_status st = CF_OK;
    for (int k = 0; k < 6 && st == CF_OK; ++k) {
        c->cur = (cur0 + k) & 1;
        c->tstep = t0 - t0 % 3 + k % 3;
        st = schedule_steps(c, n, false);
    }
    c->cur = cur0;
    c->tstep = t0;
    return st;
}

cf_status cf_synchronize(cf_ctx *c) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    return consume_errors(c);
}

cf_status cf_step(cf_ctx *c, int32_t n) {
    cf_status s = cf_step_async(c, n);
    if (s != CF_OK) return s;
    return cf_synchronize(c);
}

// True if no value of y[0..n) is an infinity or a NaN (exponent bits all
// set). Adding one unit of the exponent field to the exponent bits carries
// into the sign bit only when they are all set, so the loop is plain AND,
// ADD and OR without compares, and the compiler vectorises it (12.5 k values
// in ~2.5 us instead of ~8 us on one host core).
static bool all_finite(const double *y, long long n) {
    const uint64_t exp = 0x7ff0000000000000ull, unit = 0x0010000000000000ull;
    uint64_t bad = 0;
    for (long long i = 0; i < n; ++i) {
        uint64_t b;
        std::memcpy(&b, y + i, sizeof b);
        bad |= (b & exp) + unit;
    }
    return (bad >> 63) == 0;
}

// Device address of page-locked host memory that is mapped into the current
// device's address space, else null (pageable memory, or no mapping).
static void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not an error of the context
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cf_status cf_step_exchange(cf_ctx *c, int32_t n, const double *y_in, double *y_out) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (n < 0) return fail(c, CF_EINVAL, "n must be >= 0");
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "cf_step_exchange needs cf_lbm_init first");
    if ((y_in || y_out) && c->V == 0) return fail(c, CF_ESTATE, "no cells");
    if (y_in) {
        if (!all_finite(y_in, 3LL * c->V)) return fail(c, CF_EINVAL, "non-finite position");
        // mapped page-locked input: the conversion kernel reads it in place
        // over the host link; otherwise it is staged by a copy
        const double *src = static_cast<const double *>(mapped_host(y_in));
        if (!src) {
            CUDA_TRY(c, cudaMemcpyAsync(c->stage, y_in, sizeof(double) * 3 * c->V, cudaMemcpyHostToDevice,
                                        c->stream));
            src = c->stage;
        }
        CUDA_TRY(c, launch_set_positions(src, 0, c->V, c->xref64, c->u[c->cur], c->stream));
    }
    if (n > 0) {
        cf_status st = schedule_steps(c, n, true);
        if (st != CF_OK) return st;
    }
    if (y_out) {
        double *dst = static_cast<double *>(mapped_host(y_out));  // written in place when mapped
        CUDA_TRY(c, launch_get_positions(c->u[c->cur], c->xref64, 0, c->V, dst ? dst : c->stage, c->stream));
        if (!dst)
            CUDA_TRY(c, cudaMemcpyAsync(y_out, c->stage, sizeof(double) * 3 * c->V, cudaMemcpyDeviceToHost,
                                        c->stream));
    }
    return consume_errors(c);  // the one wait of the call
}

}  // extern "C"

namespace {

// n steps with the same kernels as cf_step, launched one after another on the
// context's stream with a CUDA event pair around every kernel, in launch
// shape sh. acc[] receives the summed milliseconds of [tet force, gather +
// spread, far LBM, near LBM (or whole-lattice LBM without cells),
// interpolation]; the state advances exactly as under cf_step(n).
cf_status timed_steps(cf_ctx *c, int n, const Shape &sh, double acc[5]) {
    const int BATCH = 32, NE = 6;
    std::vector<cudaEvent_t> ev(NE * BATCH + 2);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(c, CF_ECUDA, "event create failed");
    for (int k = 0; k < 5; ++k) acc[k] = 0.0;
    cf_status st = CF_OK;
    const MeshView m = view(c);
    const bool cells = c->T > 0;
    cudaStream_t s = c->stream;
    if (n > 0) c->macro_tile = cells ? sh.tile : -1;
    for (int done = 0; done < n && st == CF_OK;) {
        const int b = std::min(BATCH, n - done);
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < b && e == cudaSuccess; ++i) {
            const int p = c->cur, t = done + i;
            const int sph = (int)((c->tstep) % 3);
            const RegionSlot use = region_slot(c, sph), accm = accum_slot(c, sph);
            cudaEvent_t *E = &ev[NE * i];
            const RegionSlot none{nullptr};
            if (cells && t == 0) {  // region of the first step (and, with mark_k5, the next): not timed
                e = clear_slot(c, use, s);
                if (e == cudaSuccess && sh.mark_k5) e = clear_slot(c, accm, s);
                if (e == cudaSuccess) e = launch_mark_region(m, c->u[p], c->lp, use, sh.mark_k5 ? accm : none, s);
            }
            if (cells && t > 0 && sh.mark_k5 && e == cudaSuccess) e = clear_slot(c, accm, s);
            cudaEventRecord(E[0], s);
            if (cells && t > 0 && e == cudaSuccess)
                e = launch_interp_advect(m, c->vel, c->lp, c->u[1 - p], c->u[p], c->d_err, s, sh.interp_block,
                                         sh.mark_k5 ? accm : none, sh.interp_form);
            cudaEventRecord(E[1], s);
            if (cells && e == cudaSuccess) {
                if (!sh.mark_k5) e = clear_slot(c, accm, s);
                if (e == cudaSuccess && sh.fused) e = launch_chain_step(c, m, p, sh, accm, s);
                if (e == cudaSuccess && !sh.fused)
                    e = launch_tet_force(m, c->u[p], c->d_err, s, sh.tet_block, sh.tet_form,
                                         sh.mark_k5 ? nullptr : &c->lp, sh.mark_k5 ? nullptr : &accm);
            }
            cudaEventRecord(E[2], s);  // fused: the whole chain is timed as the tet-force slot
            if (cells && e == cudaSuccess && !sh.fused)
                e = launch_gather_spread(m, c->u[p], c->F, &c->lp, c->d_err, s, sh.gather_block, sh.staged);
            cudaEventRecord(E[3], s);
            if (e == cudaSuccess)
                e = cells ? launch_lbm_far(c->f[p], c->f[1 - p], c->lp, use.bits, c->seed + p, sh.far_spec, s)
                          : launch_lbm(c->f[p], c->f[1 - p], c->lp, c->seed + p, c->seed + 1 - p, s);
            cudaEventRecord(E[4], s);
            if (cells && e == cudaSuccess)
                e = launch_lbm_near(c->f[p], c->f[1 - p], c->F, c->lp, use.bits, c->vel,
                                    sh.near_rows || !c->near_tiles_fit ? 0 : near_grid(c), c->seed + p, c->seed + 1 - p, s);
            cudaEventRecord(E[5], s);
            c->cur ^= 1;
            c->tstep += 1;
        }
        if (e != cudaSuccess) {
            st = fail(c, CF_ECUDA, "launch failed: %s", cudaGetErrorString(e));
            break;
        }
        st = wait_stream(c);
        // event pairs -> [interp, tet, gather+spread, far, near]
        const int slot[5] = {4, 0, 1, 2, 3};
        for (int i = 0; i < b && st == CF_OK; ++i)
            for (int k = 0; k < 5; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[NE * i + k], ev[NE * i + k + 1]);
                acc[slot[k]] += ms;
            }
        done += b;
    }
    if (st == CF_OK && cells) {  // final K5
        const int p = c->cur ^ 1;
        cudaEventRecord(ev[NE * BATCH], s);
        cudaError_t e = launch_interp_advect(m, c->vel, c->lp, c->u[p], c->u[1 - p], c->d_err, s, sh.interp_block,
                                             RegionSlot{nullptr}, sh.interp_form);
        cudaEventRecord(ev[NE * BATCH + 1], s);
        st = e == cudaSuccess ? wait_stream(c) : fail(c, CF_ECUDA, "launch failed: %s", cudaGetErrorString(e));
        float ms = 0.f;
        if (st == CF_OK) cudaEventElapsedTime(&ms, ev[NE * BATCH], ev[NE * BATCH + 1]);
        acc[4] += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return st;
}

// Lattice nodes in the tiles of the region the last step used.
cf_status region_nodes(cf_ctx *c, long long *out) {
    *out = 0;
    if (c->T == 0 || c->tstep == 0) return CF_OK;
    const LbmParams &p = c->lp;
    const RegionSlot last = region_slot(c, (int)((c->tstep - 1) % 3));
    const size_t nw = (tiles_of(p) + 31) / 32;
    std::vector<unsigned> h(nw);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), last.bits, sizeof(unsigned) * nw, cudaMemcpyDeviceToHost, c->stream));
    cf_status st = wait_stream(c);
    if (st != CF_OK) return st;
    const int tx = 1 << p.tlx, ty = 1 << p.tly, tz = 1 << p.tlz;
    for (size_t j = 0; j < nw; ++j)
        for (unsigned w = h[j]; w; w &= w - 1u) {
            const long long t = 32 * (long long)j + __builtin_ctz(w);
            const long long ix = t % p.ntx, iy = (t / p.ntx) % p.nty, iz = t / ((long long)p.ntx * p.nty);
            const long long ex = std::min<long long>(tx, p.nx - ix * tx), ey = std::min<long long>(ty, p.ny - iy * ty),
                            ez = std::min<long long>(tz, p.nz - iz * tz);
            *out += ex * ey * ez;
        }
    return CF_OK;
}

// Device time of n coupled steps with shape sh, run exactly as cf_step(n)
// runs them (the same graphs, the two streams overlapping), the graphs
// instantiated before the timed launch. Leaves sh as the context's shape.
cf_status timed_call(cf_ctx *c, int n, const Shape &sh, double *ms) {
    c->shape = sh;
    shape_to_lbm(c->lp, sh);
    drop_graphs(c);
    cf_status st = schedule_steps(c, n, false);
    if (st != CF_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    if (e == cudaSuccess) {
        st = schedule_steps(c, n, true);
        if (st == CF_OK) e = cudaEventRecord(e1, c->stream);
    }
    if (e == cudaSuccess && st == CF_OK) {
        st = wait_stream(c);
        float t = 0.f;
        if (st == CF_OK) e = cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != CF_OK) return st;
    if (e != cudaSuccess) return fail(c, CF_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
    return consume_errors(c);
}

}  // namespace

extern "C" {

cf_status cf_step_profiled(cf_ctx *c, int32_t n, double *kernel_ms, int64_t *near_nodes) {
    if (!c || !kernel_ms) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (n < 1) return fail(c, CF_EINVAL, "n must be >= 1");
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "cf_step needs cf_lbm_init first");
    double acc[5];
    cf_status st = timed_steps(c, n, c->shape, acc);
    if (st == CF_OK && near_nodes) {
        long long nn = 0;
        st = region_nodes(c, &nn);
        *near_nodes = nn;
    }
    if (st != CF_OK) return st;
    for (int k = 0; k < 5; ++k) kernel_ms[k] = acc[k] / n;
    return consume_errors(c);
}

cf_status cf_get_launch_shape(cf_ctx *c, int32_t *shape) {
    if (!c || !shape) return CF_EINVAL;
    const Shape &sh = c->shape;
    shape[0] = 1 << kTileShapes[sh.tile][0];
    shape[1] = 1 << kTileShapes[sh.tile][1];
    shape[2] = 1 << kTileShapes[sh.tile][2];
    shape[3] = sh.tet_block;
    shape[4] = sh.gather_block;
    shape[5] = sh.interp_block;
    shape[6] = sh.fused;
    shape[7] = sh.near_rows;
    shape[8] = sh.far_spec;
    shape[9] = sh.tet_form;
    shape[10] = sh.pop_l2;
    shape[11] = sh.pop_pairs;
    shape[12] = sh.mark_k5;
    shape[13] = sh.staged;
    shape[14] = sh.interp_form;
    return CF_OK;
}

cf_status cf_set_launch_shape(cf_ctx *c, const int32_t *shape) {
    if (!c || !shape) return CF_EINVAL;
    DeviceGuard dg(c->device);
    Shape sh;
    sh.tile = -1;
    for (int k = 0; k < kNumTileShapes; ++k)
        if (shape[0] == 1 << kTileShapes[k][0] && shape[1] == 1 << kTileShapes[k][1] &&
            shape[2] == 1 << kTileShapes[k][2])
            sh.tile = k;
    if (sh.tile < 0)
        return fail(c, CF_EINVAL, "tile %dx%dx%d is not one of 16x4x4, 32x4x2, 32x2x4, 8x8x4", shape[0], shape[1],
                    shape[2]);
    for (int k = 3; k < 6; ++k)
        if (shape[k] < 32 || shape[k] > 256 || shape[k] % 32)
            return fail(c, CF_EINVAL, "block size %d: need a multiple of 32 in [32, 256]", shape[k]);
    sh.tet_block = shape[3];
    sh.gather_block = shape[4];
    sh.interp_block = shape[5];
    if (shape[6] != 0 && shape[6] != 1) return fail(c, CF_EINVAL, "fused must be 0 or 1");
    sh.fused = shape[6];
    if (shape[7] != 0 && shape[7] != 1) return fail(c, CF_EINVAL, "near_rows must be 0 or 1");
    sh.near_rows = shape[7];
    if (shape[8] != 0 && shape[8] != 1) return fail(c, CF_EINVAL, "far_spec must be 0 or 1");
    sh.far_spec = shape[8];
    if (shape[9] < 0 || shape[9] > 2) return fail(c, CF_EINVAL, "tet_form must be 0, 1 or 2");
    sh.tet_form = shape[9];
    if (shape[10] != 0 && shape[10] != 1) return fail(c, CF_EINVAL, "pop_l2 must be 0 or 1");
    sh.pop_l2 = shape[10];
    if (shape[11] != 0 && shape[11] != 1) return fail(c, CF_EINVAL, "pop_pairs must be 0 or 1");
    sh.pop_pairs = shape[11];
    if (shape[12] != 0 && shape[12] != 1) return fail(c, CF_EINVAL, "mark_k5 must be 0 or 1");
    sh.mark_k5 = shape[12];
    if (shape[13] != 0 && shape[13] != 1) return fail(c, CF_EINVAL, "staged must be 0 or 1");
    sh.staged = shape[13];
    if (shape[14] != 0 && shape[14] != 1) return fail(c, CF_EINVAL, "interp_form must be 0 or 1");
    sh.interp_form = shape[14];
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // no graph of the old shape in flight
    drop_graphs(c);
    c->shape = sh;
    if (c->lbm_ready) shape_to_lbm(c->lp, sh);
    return CF_OK;
}

cf_status cf_set_chain_wait(cf_ctx *c, int64_t max_polls, int32_t extra_need) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (max_polls < 1 || extra_need < 0) return fail(c, CF_EINVAL, "need max_polls >= 1 and extra_need >= 0");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // no graph with the old arguments in flight
    drop_graphs(c);
    c->chain_spin_limit = max_polls;
    c->chain_extra_need = extra_need;
    return c->cells.empty() ? CF_OK : build_chain_items(c);
}

cf_status cf_autotune(cf_ctx *c, int32_t steps_per_candidate, int32_t *shape_out) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (steps_per_candidate < 1) return fail(c, CF_EINVAL, "steps_per_candidate must be >= 1");
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "cf_autotune needs cf_lbm_init first");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->T > 0) {
        // one knob at a time, the others at their best so far; a candidate
        // is rated by the time of whole pipelined steps, so that what the
        // far field overlaps counts as it does in cf_step
        struct Knob {
            int Shape::*field;
            std::vector<int> cands;
        };
        const Knob knobs[] = {
            {&Shape::tile, {0, 1, 2, 3}},
            {&Shape::fused, {0, 1}},
            {&Shape::near_rows, {0, 1}},
            {&Shape::far_spec, {0, 1}},
            {&Shape::tet_form, {0, 1, 2}},
            {&Shape::pop_l2, {0, 1}},
            {&Shape::pop_pairs, {1, 0}},
            {&Shape::mark_k5, {0, 1}},
            {&Shape::staged, {0, 1}},
            {&Shape::interp_form, {0, 1}},
            {&Shape::tet_block, {64, 128, 256}},
            {&Shape::gather_block, {64, 128, 256}},
            {&Shape::interp_block, {64, 128, 256}},
        };
        const Shape start = c->shape;
        Shape best = start;
        for (const Knob &k : knobs) {
            double tbest = 1e300;
            int vbest = best.*k.field;
            for (int v : k.cands) {
                Shape sh = best;
                sh.*k.field = v;
                double t = 0.0;
                const cf_status st = timed_call(c, steps_per_candidate, sh, &t);
                if (st != CF_OK) {
                    c->shape = start;
                    shape_to_lbm(c->lp, start);
                    drop_graphs(c);
                    return st;
                }
                if (t < tbest) {
                    tbest = t;
                    vbest = v;
                }
            }
            best.*k.field = vbest;
        }
        c->shape = best;
        shape_to_lbm(c->lp, best);
        drop_graphs(c);
    }
    return shape_out ? cf_get_launch_shape(c, shape_out) : CF_OK;
}

cf_status cf_compute_forces(cf_ctx *c) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (c->T == 0) return fail(c, CF_ESTATE, "no cells");
    const MeshView m = view(c);
    CUDA_TRY(c, launch_tet_force(m, c->u[c->cur], c->d_err, c->stream));
    CUDA_TRY(c, launch_gather_spread(m, c->u[c->cur], nullptr, nullptr, c->d_err, c->stream));
    return consume_errors(c);
}

cf_status cf_get_forces(cf_ctx *c, int32_t id, double *out) {
    int v0, nv;
    if (!vertex_range(c, id, &v0, &nv) || !out) return fail(c, CF_EINVAL, "unknown cell or null output");
    DeviceGuard dg(c->device);
    CUDA_TRY(c, launch_get_forces(c->fv, v0, nv, c->stage, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->stage, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

cf_status cf_get_positions(cf_ctx *c, int32_t id, double *out) {
    int v0, nv;
    if (!vertex_range(c, id, &v0, &nv) || !out) return fail(c, CF_EINVAL, "unknown cell or null output");
    DeviceGuard dg(c->device);
    CUDA_TRY(c, launch_get_positions(c->u[c->cur], c->xref64, v0, nv, c->stage, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->stage, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

cf_status cf_set_positions(cf_ctx *c, int32_t id, const double *y) {
    int v0, nv;
    if (!vertex_range(c, id, &v0, &nv) || !y) return fail(c, CF_EINVAL, "unknown cell or null input");
    DeviceGuard dg(c->device);
    if (!all_finite(y, 3LL * nv)) return fail(c, CF_EINVAL, "non-finite position");
    CUDA_TRY(c, cudaMemcpyAsync(c->stage, y, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_set_positions(c->stage, v0, nv, c->xref64, c->u[c->cur], c->stream));
    return wait_stream(c);
}

static cf_status get_macro(cf_ctx *c, double *rho_out, double *u_out) {
    if (!c) return CF_EINVAL;
    DeviceGuard dg(c->device);
    if (!c->lbm_ready) return fail(c, CF_ESTATE, "no fluid: call cf_lbm_init");
    const size_t N = (size_t)c->lp.N;
    double *d;
    CUDA_TRY(c, dalloc(&d, u_out ? 3 * N : N));
    // the last step's force region, in the tiling that step ran with
    LbmParams q = c->lp;
    const unsigned *bits = nullptr;
    if (c->macro_tile >= 0 && c->tstep > 0) {
        set_tiles(q, c->macro_tile);
        bits = region_slot(c, (int)((c->tstep - 1) % 3)).bits;
    }
    cudaError_t e = launch_lbm_macro(c->f[c->cur], c->F, q, bits, c->vel, u_out ? nullptr : d, u_out ? d : nullptr,
                                     c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u_out ? u_out : rho_out, d, sizeof(double) * (u_out ? 3 * N : N), cudaMemcpyDeviceToHost,
                            c->stream);
    cf_status s = e == cudaSuccess ? wait_stream(c) : fail(c, CF_ECUDA, "%s", cudaGetErrorString(e));
    cudaFree(d);
    return s;
}

cf_status cf_get_velocity(cf_ctx *c, double *out) {
    if (!out) return fail(c, CF_EINVAL, "null output");
    return get_macro(c, nullptr, out);
}

cf_status cf_get_density(cf_ctx *c, double *out) {
    if (!out) return fail(c, CF_EINVAL, "null output");
    return get_macro(c, out, nullptr);
}

cf_status cf_get_energy(cf_ctx *c, int32_t id, double *out) {
    const CellInfo *ci = cell_of(c, id);
    if (!ci || !out) return fail(c, CF_EINVAL, "unknown cell or null output");
    DeviceGuard dg(c->device);
    CUDA_TRY(c, launch_energy(view(c), c->u[c->cur], ci->t_off, ci->t_off + ci->nt, c->energy_partial, c->energy_out,
                              c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->energy_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

cf_status cf_get_taylor(cf_ctx *c, int32_t id, double *out) {
    const CellInfo *ci = cell_of(c, id);
    if (!ci || !out) return fail(c, CF_EINVAL, "unknown cell or null output");
    DeviceGuard dg(c->device);
    CUDA_TRY(c, launch_taylor(view(c), c->u[c->cur], ci->t_off, ci->t_off + ci->nt, c->taylor_partial, c->taylor_out,
                              c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->taylor_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return wait_stream(c);
}

cf_status cf_get_cell_strain(cf_ctx *c, int32_t id, double d_ref, double *out) {
    const CellInfo *ci = cell_of(c, id);
    if (!ci || !out) return fail(c, CF_EINVAL, "unknown cell or null output");
    if (!(d_ref > 0.0) || !std::isfinite(d_ref)) return fail(c, CF_EINVAL, "d_ref must be positive and finite");
    DeviceGuard dg(c->device);
    unsigned *word = reinterpret_cast<unsigned *>(c->d_status);  // device scratch of the context
    CUDA_TRY(c, launch_max_extent(view(c), c->u[c->cur], ci->v_off, ci->nv, word, c->stream));
    unsigned bits = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&bits, word, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    const cf_status s = wait_stream(c);
    if (s != CF_OK) return s;
    float d2;
    std::memcpy(&d2, &bits, sizeof d2);
    out[0] = std::sqrt((double)d2);
    out[1] = (out[0] - d_ref) / d_ref;
    return CF_OK;
}

cf_status cf_get_csr(cf_ctx *c, int32_t id, int32_t *ptr, int32_t *idx) {
    const CellInfo *ci = cell_of(c, id);
    if (!ci || !ptr || !idx) return fail(c, CF_EINVAL, "unknown cell or null output");
    DeviceGuard dg(c->device);
    std::vector<int> p(ci->nv + 1);
    CUDA_TRY(c, cudaMemcpyAsync(p.data(), c->csr_ptr + ci->v_off, sizeof(int) * (ci->nv + 1), cudaMemcpyDeviceToHost,
                                c->stream));
    cf_status s = wait_stream(c);
    if (s != CF_OK) return s;
    const int base = p[0], len = p[ci->nv] - p[0];
    if (len != 4 * ci->nt) return fail(c, CF_ECUDA, "incidence rows inconsistent");
    CUDA_TRY(c, cudaMemcpyAsync(idx, c->csr_idx + base, sizeof(int) * len, cudaMemcpyDeviceToHost, c->stream));
    s = wait_stream(c);
    if (s != CF_OK) return s;
    for (int v = 0; v <= ci->nv; ++v) ptr[v] = p[v] - base;
    for (int e = 0; e < len; ++e) idx[e] -= 4 * ci->t_off;
    return CF_OK;
}

cf_status cf_get_mesh(cf_ctx *c, int32_t id, int32_t *tets, double *B, double *V0) {
    const CellInfo *ci = cell_of(c, id);
    if (!ci) return fail(c, CF_EINVAL, "unknown cell");
    DeviceGuard dg(c->device);
    const int nt = ci->nt, T = c->T;
    if (tets) {
        std::vector<int4> t(nt);
        CUDA_TRY(c, cudaMemcpyAsync(t.data(), c->tet + ci->t_off, sizeof(int4) * nt, cudaMemcpyDeviceToHost, c->stream));
        cf_status s = wait_stream(c);
        if (s != CF_OK) return s;
        for (int i = 0; i < nt; ++i) {
            tets[4 * i] = t[i].x - ci->v_off;
            tets[4 * i + 1] = t[i].y - ci->v_off;
            tets[4 * i + 2] = t[i].z - ci->v_off;
            tets[4 * i + 3] = t[i].w - ci->v_off;
        }
    }
    if (B) {
        std::vector<float> b(9 * (size_t)nt);
        CUDA_TRY(c, cudaMemcpy2DAsync(b.data(), sizeof(float) * nt, c->B + ci->t_off, sizeof(float) * T,
                                      sizeof(float) * nt, 9, cudaMemcpyDeviceToHost, c->stream));
        cf_status s = wait_stream(c);
        if (s != CF_OK) return s;
        for (int i = 0; i < nt; ++i)
            for (int k = 0; k < 9; ++k) B[9 * i + k] = b[(size_t)k * nt + i];
    }
    if (V0) {
        std::vector<float> v(nt);
        CUDA_TRY(c, cudaMemcpyAsync(v.data(), c->V0 + ci->t_off, sizeof(float) * nt, cudaMemcpyDeviceToHost, c->stream));
        cf_status s = wait_stream(c);
        if (s != CF_OK) return s;
        for (int i = 0; i < nt; ++i) V0[i] = v[i];
    }
    return CF_OK;
}

int32_t cf_cell_verts(const cf_ctx *c, int32_t id) {
    if (c && id == CF_ALL_CELLS) return c->V;
    return (c && id >= 0 && id < (int)c->cells.size()) ? c->cells[id].nv : 0;
}

int32_t cf_cell_tets(const cf_ctx *c, int32_t id) {
    if (c && id == CF_ALL_CELLS) return c->T;
    return (c && id >= 0 && id < (int)c->cells.size()) ? c->cells[id].nt : 0;
}

}  // extern "C"
