// Internal declarations of the GB300 cell/fluid library: device layouts,
// kernel launchers and the D3Q19 lattice as compile-time constants.
//
// Device layout (structure of arrays for the streams that consecutive
// threads read word by word; float4 per node or vertex where a thread reads
// all three components of one point):
//   populations  f[q * N + n], q = 0..18, n = x + nx*(y + ny*z), stored as the
//                deviation f_q - w_q from the rest equilibrium (keeps FP32
//                rounding relative to the O(u) signal, not to O(w_q));
//   force field  float4 F[n] = (Fx, Fy, Fz, 0): one vector atomic per node
//                in the spread, one 16-byte load in the near field; with the
//                deterministic spread the same buffer holds long long
//                Fi[3][N], the components in fixed point (units of 2^-48):
//                integer additions are exact and independent of their order;
//   u(t)         float4 vel[n] = (ux, uy, uz, 0) on the force region (one
//                16-byte load per support node in the interpolation);
//   vertices     float4 per vertex (one 16-byte load in the tet gathers):
//                xr (FP32 x_ref relative to the cell's integer origin, .w =
//                cell id), u (FP32 displacement y - x_ref), fv (force);
//                xref64 [V][3] FP64 for exact host round trips;
//   tets         int4 tet[t], B[(3k + j) * T + t] (FP32, and FP64 in B64), V0[t],
//                tcell[t];
//   corner force float4 fc[c * T + t].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#ifdef __CUDACC__
#include <cooperative_groups.h>
#endif

namespace cf {

// Error bits of the device error word (never trapped; read by the host).
enum : unsigned {
    ERR_INVERTED = 1u << 0,   // det F <= 0 in some tet
    ERR_NONFINITE = 1u << 1,  // NaN / Inf in a force or a displacement
    ERR_DOMAIN = 1u << 2,     // delta support outside 0 <= y <= ny-1
    ERR_MOVED = 1u << 3,      // a support node fell outside the step's force region
    ERR_WAIT = 1u << 4,       // a bounded wait of the fused cell chain gave up
};

// ---------------------------------------------------------------- D3Q19
// Velocity set: q = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the twelve
// vectors with two nonzero components in lexicographic order of (cx,cy,cz).
// Opposite of q: axis pairs swap within (1,2), (3,4), (5,6); diagonal q <-> 25-q.
__host__ __device__ constexpr int cx(int q) {
    return q == 1 ? 1 : q == 2 ? -1 : (q >= 7 && q <= 10) ? -1 : (q >= 15) ? 1 : 0;
}
__host__ __device__ constexpr int cy(int q) {
    return q == 3 ? 1 : q == 4 ? -1
         : (q == 7 || q == 11 || q == 12 || q == 15) ? -1
         : (q == 10 || q == 13 || q == 14 || q == 18) ? 1 : 0;
}
__host__ __device__ constexpr int cz(int q) {
    return q == 5 ? 1 : q == 6 ? -1
         : (q == 8 || q == 11 || q == 13 || q == 16) ? -1
         : (q == 9 || q == 12 || q == 14 || q == 17) ? 1 : 0;
}
__host__ __device__ constexpr int opp(int q) {
    return q == 0 ? 0 : q <= 6 ? (q % 2 ? q + 1 : q - 1) : 25 - q;
}
__host__ __device__ constexpr float wq(int q) {
    return q == 0 ? 1.0f / 3.0f : q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f;
}

// Population storage formats (see csrc/lbm.cu).
enum : int { POP_F32 = 0, POP_F16 = 1, POP_BF16 = 2 };

struct LbmParams {
    int fmt;  // POP_F32, POP_F16 or POP_BF16
    int sr;   // 16-bit stores rounded stochastically (else to nearest)
    int nx, ny, nz;
    long long N;
    float omega;        // 1/tau
    float guo;          // 1 - 1/(2 tau)
    float uw_lo, uw_hi; // wall x velocities at y = -1/2 and y = ny - 1/2
    float gx, gy, gz;   // uniform body-force density
    int dw;             // delta kernel: support width 2 (trilinear) or 4 (Peskin)
    int l2;             // FP32 far and near fields: populations cached in L2 at normal priority
                        // (1) instead of streamed with evict-first hints (0)
    int pairs;          // 16-bit formats, nx even: two nodes per thread in the row-form kernels
    int det;            // deterministic spread: the force field in fixed point, long long [3][N]
    // force-region tiles of 2^tlx x 2^tly x 2^tlz = 256 nodes (x fastest;
    // the last tile of an axis may stick out of the lattice), ntx * nty * ntz
    // of them
    int tlx, tly, tlz;
    int ntx, nty, ntz;
};

struct MeshView {
    int V, T;
    const float4 *xr;      // [V]: x_ref - origin (FP32), .w = cell id (int bits)
    const int *origin;     // [3 * ncells], integer origin of each cell
    const int4 *tet;       // [T]: global vertex indices, corner 3 = vertex 4
    const float *B;        // [9][T]: B[(3k + j) * T + t] = (J^-1)_kj
    const double *B64;     // [9][T] or null: the same in FP64 (J - 1 of nearly incompressible tets)
    const float4 *Bp;      // [3][T] or null: row k of B with .w = V0, cell id (int bits), 0 for k = 0, 1, 2
    const float *V0;       // [T]
    const int *tcell;      // [T]: cell of each tet
    const int *tmat;       // [T] or null: material slot of each tet (null: the cell's slot, = cell id)
    const float4 *mat;     // [ncells]: mu1, mu2, kappa, w
    const int *csr_ptr;    // [V+1]
    const int *csr_idx;    // [4T]: entries 4 t + c, ascending per row
    float4 *fc;            // [4][T]: corner force fc[c * T + t]
    float4 *fv;            // [V]: vertex force
};

// Delta kernels delta_h(r) = phi(r_x) phi(r_y) phi(r_z) of support width W
// (nodes per axis):
//   W = 2, trilinear:  phi(r) = max(0, 1 - |r|);
//   W = 4, Peskin's four-point kernel (C. S. Peskin, The immersed boundary
//          method, Acta Numerica 11, 2002, Sec. 6):
//          phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2)) / 8   for |r| <= 1,
//                   (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2)) / 8  for 1 <= |r| <= 2,
//                   0 beyond.
// The support of a point p on one axis is the W nodes lo + k, k = 0..W-1,
// with lo = floor(p) - (W/2 - 1). Shared by the spread, the interpolation
// and the region marking so that all three see exactly the same node set.
struct Support {
    int bx, by, bz;     // lower corner lo (absolute node, x and z not yet wrapped)
    float fx, fy, fz;   // p - floor(p) per axis, in [0, 1)
};

// False if the position is not finite, absurdly far away, or the support
// leaves 0 <= y <= ny-1.
template <int W>
__device__ __forceinline__ bool support_of(const int *__restrict__ origin, float4 xr, float4 u, int ny, Support &s) {
    const int c = __float_as_int(xr.w);
    const float px = xr.x + u.x, py = xr.y + u.y, pz = xr.z + u.z;
    if (!(fabsf(px) < 1e6f && fabsf(py) < 1e6f && fabsf(pz) < 1e6f)) return false;  // also NaN
    const float lx = floorf(px), ly = floorf(py), lz = floorf(pz);
    s.fx = px - lx;
    s.fy = py - ly;
    s.fz = pz - lz;
    s.bx = (int)lx + __ldg(origin + 3 * c + 0) - (W / 2 - 1);
    s.by = (int)ly + __ldg(origin + 3 * c + 1) - (W / 2 - 1);
    s.bz = (int)lz + __ldg(origin + 3 * c + 2) - (W / 2 - 1);
    return s.by >= 0 && s.by + W - 1 <= ny - 1;
}

// One-axis weights phi(p - (lo + k)), k = 0..W-1, from f = p - floor(p).
// For W = 4 the distances are 1 + f, f, 1 - f, 2 - f, and both branches of
// phi reduce to the same root q = sqrt(1 + 4f - 4f^2).
template <int W>
__device__ __forceinline__ void delta_weights(float f, float (&w)[W]);
template <>
__device__ __forceinline__ void delta_weights<2>(float f, float (&w)[2]) {
    w[0] = 1.f - f;
    w[1] = f;
}
// Every operation is rounded explicitly (no contraction), so the weights
// are the same bits wherever they are inlined.
template <>
__device__ __forceinline__ void delta_weights<4>(float f, float (&w)[4]) {
    const float q = __fsqrt_rn(__fmaf_rn(__fmul_rn(4.f, f), __fsub_rn(1.f, f), 1.f));
    const float a = __fsub_rn(3.f, __fmul_rn(2.f, f)), b = __fadd_rn(1.f, __fmul_rn(2.f, f));
    w[0] = __fmul_rn(0.125f, __fsub_rn(a, q));
    w[1] = __fmul_rn(0.125f, __fadd_rn(a, q));
    w[2] = __fmul_rn(0.125f, __fadd_rn(b, q));
    w[3] = __fmul_rn(0.125f, __fsub_rn(b, q));
}

// ---------------------------------------------------------------- force field access
// The force field is float4 per node, or (p.det) fixed point: component k of
// node n is the integer Fi[k * N + n] in units of 2^-48. A contribution is
// converted by one rounding of its FP32 value scaled by 2^48 (exact for
// values above 2^-24 in magnitude, which FP32 already carries at that
// resolution); the sum of the integers is exact whatever the order of the
// atomics, so every run, launch shape and schedule spreads the same field.
// |F| must stay below 2^15 per component (far beyond any stable run).
constexpr float kFixScale = 281474976710656.0f;  // 2^48
constexpr double kFixUnit = 1.0 / 281474976710656.0;

#ifdef __CUDACC__
__device__ __forceinline__ void force_add(float4 *F, const LbmParams &p, long long n, float ax, float ay, float az) {
    if (p.det) {
        unsigned long long *Fi = reinterpret_cast<unsigned long long *>(F);
        atomicAdd(Fi + n, (unsigned long long)__float2ll_rn(ax * kFixScale));
        atomicAdd(Fi + p.N + n, (unsigned long long)__float2ll_rn(ay * kFixScale));
        atomicAdd(Fi + 2 * p.N + n, (unsigned long long)__float2ll_rn(az * kFixScale));
    } else {
        atomicAdd(F + n, make_float4(ax, ay, az, 0.f));
    }
}

// The force at node n (read through L2); *nonzero tells whether any component is.
__device__ __forceinline__ float4 force_at(const float4 *F, const LbmParams &p, long long n, bool &nonzero) {
    if (p.det) {
        const long long *Fi = reinterpret_cast<const long long *>(F);
        const long long x = __ldcg(Fi + n), y = __ldcg(Fi + p.N + n), z = __ldcg(Fi + 2 * p.N + n);
        nonzero = (x | y | z) != 0;
        return make_float4((float)((double)x * kFixUnit), (float)((double)y * kFixUnit), (float)((double)z * kFixUnit),
                           0.f);
    }
    const float4 a = __ldcg(F + n);
    nonzero = a.x != 0.f || a.y != 0.f || a.z != 0.f;
    return a;
}

__device__ __forceinline__ void force_clear(float4 *F, const LbmParams &p, long long n) {
    if (p.det) {
        long long *Fi = reinterpret_cast<long long *>(F);
        Fi[n] = 0;
        Fi[p.N + n] = 0;
        Fi[2 * p.N + n] = 0;
    } else {
        F[n] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
#endif

__host__ __device__ __forceinline__ int wrapi(int i, int n) {
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Force region of a step: the set of tiles that hold a node that may carry
// force in that step, as a bitset over the tiles. A step's region holds every
// tile that meets the delta support of a vertex grown by one node per side
// (a vertex moves less than one spacing per step, so the support at the next
// step stays inside). Nodes outside the region see no force.
constexpr int kTileNodes = 256;

struct RegionSlot {
    unsigned *bits;  // [ceil(tiles / 32)]
};

__host__ __device__ __forceinline__ bool region_has(const unsigned *__restrict__ bits, int t) {
    return (bits[t >> 5] >> (t & 31)) & 1u;
}

// Add tile t: an atomic OR whose result is not used (a reduction the thread
// does not wait for), skipped for the (many) tiles whose bit a plain read
// already shows (a stale L1 line can only miss a bit set during this launch,
// which costs one redundant reduction).
__device__ __forceinline__ void region_add(const RegionSlot &r, int t) {
    const unsigned bit = 1u << (t & 31);
    if (r.bits[t >> 5] & bit) return;
    atomicOr(r.bits + (t >> 5), bit);
}

__host__ __device__ __forceinline__ int tile_index(const LbmParams &p, int tx, int ty, int tz) {
    return (tz * p.nty + ty) * p.ntx + tx;
}

// Tiles met by the node range [lo, hi] on one axis: the first tile t0 and
// the count; tiles are t0, t0 + 1, ... modulo nt (a periodic range wraps
// from the last tile to tile 0). `periodic` false: lo and hi already lie in
// [0, n).
struct TileRange {
    int t0, cnt;
};

__host__ __device__ __forceinline__ TileRange tile_range(int lo, int hi, int n, int lg, int nt, bool periodic) {
    TileRange r;
    if (!periodic || (lo >= 0 && hi < n)) {  // no wrap
        r.t0 = lo >> lg;
        r.cnt = (hi >> lg) - r.t0 + 1;
        return r;
    }
    if (hi - lo + 1 >= n) {
        r.t0 = 0;
        r.cnt = nt;
        return r;
    }
    const int lw = wrapi(lo, n), hw = wrapi(hi, n);
    r.t0 = lw >> lg;
    const int t1 = hw >> lg;
    if (hw >= lw) {
        r.cnt = t1 - r.t0 + 1;
    } else {  // crosses the seam: t0 .. nt-1, then 0 .. t1
        r.cnt = t1 - r.t0 + nt + 1;
        if (r.cnt > nt) r.cnt = nt;
    }
    return r;
}

// The tiles met by the node box [x0,x1] x [y0,y1] x [z0,z1] (x and z
// unwrapped, y clamped to the lattice by the caller): n of them, the k-th
// (x fastest) given by tile_of_box.
struct TileBox {
    TileRange rx, ry, rz;
    int n;
};

__host__ __device__ __forceinline__ TileBox tile_box(const LbmParams &p, int x0, int x1, int y0, int y1, int z0,
                                                     int z1) {
    TileBox b;
    b.rx = tile_range(x0, x1, p.nx, p.tlx, p.ntx, true);
    b.ry = tile_range(y0, y1, p.ny, p.tly, p.nty, false);
    b.rz = tile_range(z0, z1, p.nz, p.tlz, p.ntz, true);
    b.n = b.rx.cnt * b.ry.cnt * b.rz.cnt;
    return b;
}

__host__ __device__ __forceinline__ int tile_of_box(const LbmParams &p, const TileBox &b, int k) {
    const int r = k / b.rx.cnt;
    int tx = b.rx.t0 + (k - r * b.rx.cnt);
    tx -= tx >= p.ntx ? p.ntx : 0;
    int tz = b.rz.t0 + r / b.ry.cnt;
    tz -= tz >= p.ntz ? p.ntz : 0;
    return tile_index(p, tx, b.ry.t0 + r % b.ry.cnt, tz);
}

// Visit the tiles of the box, each once.
template <class Fn>
__host__ __device__ __forceinline__ void for_each_tile(const LbmParams &p, int x0, int x1, int y0, int y1, int z0, int z1,
                                              Fn &&fn) {
    const TileBox b = tile_box(p, x0, x1, y0, y1, z0, z1);
    for (int k = 0; k < b.n; ++k) fn(tile_of_box(p, b, k));
}

#ifdef __CUDACC__
// Add the tiles of the force region around one vertex: its support grown by
// one node per side (y clamped to the lattice). `nlanes` lanes may share a
// vertex, lane `lane` taking the tiles lane, lane + nlanes, ... of its box,
// so that a vertex's tiles are added in parallel rather than one after
// another. Neighbouring vertices mostly meet the same tiles, so the lanes of
// a warp that hold the same tile at the same step elect one of them to add
// it: a region slot has few words, and one atomic per warp and tile, instead
// of one per lane, keeps them from serialising.
template <int W>
__device__ __forceinline__ void mark_region(const Support &s, const LbmParams &p, const RegionSlot &r, int lane = 0,
                                            int nlanes = 1) {
    namespace cg = cooperative_groups;
    const TileBox b = tile_box(p, s.bx - 1, s.bx + W, max(s.by - 1, 0), min(s.by + W, p.ny - 1), s.bz - 1, s.bz + W);
    for (int k = lane; k < b.n; k += nlanes) {
        const int t = tile_of_box(p, b, k);
        const cg::coalesced_group same = cg::labeled_partition(cg::coalesced_threads(), t);
        if (same.thread_rank() == 0) region_add(r, t);
    }
}
#endif

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return the launch status.
// Once per cell (Sec. 3.2): validate, orient, B = J^-1 and V_0 in FP64;
// *status receives min over failing tets of ((t_report + t) << 8 | code),
// code 1 = index out of range, 2 = repeated vertex, 3 = degenerate.
cudaError_t launch_mesh_prepare(const double *x64, int nv, const int *tets_in, int nt, int v_off, int t_off,
                                int t_report, int T, int cell, int4 *tet, float *B, double *B64, float *V0,
                                int *tcell, unsigned long long *status, cudaStream_t s);
cudaError_t launch_vertex_prepare(const double *x64, const double *y64, int nv, int v_off, int cell,
                                  const int *origin_host3, float4 *xr, float4 *u0, float4 *u1, double *xref64,
                                  cudaStream_t s);
cudaError_t launch_csr_build(const int4 *tet, int T, int V, int *ptr, int *idx, int *cursor, cudaStream_t s);
// Packed per-tet rows for the force kernel: Bp[k * T + t] = (B_k0, B_k1, B_k2, w_k), w = (V0, material slot, 0).
cudaError_t launch_pack_tets(int T, const float *B, const float *V0, const int *tmat, float4 *Bp, cudaStream_t s);
// tmat[t] += delta where tmat[t] >= from, t < T (material slots move up when cells are added).
cudaError_t launch_shift_slots(int T, int from, int delta, int *tmat, cudaStream_t s);
cudaError_t launch_set_positions(const double *y64, int v0, int nv, const double *xref64, float4 *u,
                                 cudaStream_t s);
cudaError_t launch_get_positions(const float4 *u, const double *xref64, int v0, int nv, double *y64,
                                 cudaStream_t s);
cudaError_t launch_get_forces(const float4 *fv, int v0, int nv, double *out, cudaStream_t s);

// K1: elastic corner forces of all tets at displacements u. form 0: one
// thread per tet; 1: two tets per thread (both tets' loads issued before
// either is computed); 2: four lanes per tet (needs the packed rows m.Bp,
// else one thread per tet). With lp and mark_out non-null the same launch
// also runs one thread per vertex (blocks at the front) that adds the
// tiles of the next step's force region (the support of x + u grown by one
// node) to mark_out.
cudaError_t launch_tet_force(const MeshView &m, const float4 *u, unsigned *err, cudaStream_t s, int block = 0,
                             int form = 0, const LbmParams *lp = nullptr, const RegionSlot *mark_out = nullptr);
// Per-tet V_0 U of tets [t0, t1) reduced in a fixed order into *out (double).
cudaError_t launch_energy(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s);
// K8: Taylor deformation of tets [t0, t1) at displacements u; out[10] (device)
// = D, D from the printed squared expression, inclination (deg), a1, a2, a3,
// theta1, theta2, theta3, volume. partial: 10 doubles per 256 tets.
// Squared largest distance between two of the vertices [v0, v0 + nv) at
// displacements u, as the bits of a float in *out (device).
cudaError_t launch_max_extent(const MeshView &m, const float4 *u, int v0, int nv, unsigned *out, cudaStream_t s);
cudaError_t launch_taylor(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s);
// K2 (+K3): vertex force sums over the incidence rows; with F != null the
// same threads spread their vertex force onto the lattice, directly with
// global atomics or (staged) through a shared-memory box per block of
// vertices.
cudaError_t launch_gather_spread(const MeshView &m, const float4 *u, float4 *F, const LbmParams *lp, unsigned *err,
                                 cudaStream_t s, int block = 0, int staged = 0);
// Shared-memory opt-in of the staged spread (once per context, before any
// capture).
cudaError_t prepare_staged_spread();
// Add the force region of the positions x + u (support grown by one node) to
// a region slot, and to a second one if r2.bits is not null (both cleared by
// the caller).
cudaError_t launch_mark_region(const MeshView &m, const float4 *u, const LbmParams &p, const RegionSlot &r,
                               const RegionSlot &r2, cudaStream_t s);
// K1 + K23 fused (csrc/chain.cu): one persistent launch that runs the work
// items of the cell chain in order: items[i] = (kind, cell, begin, end) with
// kind 0 = region marking of vertices [begin, end) into mark (skipped when
// mark.bits is null), 1 = corner forces of tets [begin, end) of `cell`, 2 =
// vertex sums + spread of vertices [begin, end) of `cell`. A kind-2 item
// waits until the need[cell] kind-1 items of its cell are done, giving up
// after spin_limit polls (ERR_WAIT); counters[2 + ncells] must be zero at
// launch.
cudaError_t launch_cell_chain(const MeshView &m, const float4 *u, float4 *F, const LbmParams &lp,
                              const RegionSlot &mark, unsigned *err, const int4 *items, int nitems, const int *need,
                              int *counters, int blocks, long long spin_limit, cudaStream_t s);
// K4: pull stream + BGK collide with Guo forcing, fin -> fout, every node, no
// force field (fluid-only runs). Population buffers are in the format p.fmt.
// Every stream-collide launch reads the step's rounding seed from seed[0];
// the launch that closes a step (this one, or the near field) stores
// seed[0] + 1 into next_seed (the seed of the other buffer parity).
cudaError_t launch_lbm(const void *fin, void *fout, const LbmParams &p, const unsigned *seed, unsigned *next_seed,
                       cudaStream_t s);
// K4 split by the force region: far = the nodes outside it (rows of 128
// nodes; threads in region tiles return at once), with no force-field read;
// near = the region's tiles (blocks stride over the set bits of its
// bitset), with the force field, also storing u(t) there; it zeroes the
// force field where it read a nonzero one, so that F is zero everywhere
// between steps. spec: the far field issues a node's loads before its
// region test resolves.
cudaError_t launch_lbm_far(const void *fin, void *fout, const LbmParams &p, const unsigned *bits,
                           const unsigned *seed, bool spec, cudaStream_t s);
// blocks > 0: that many blocks stride over the region's tiles (the set bits
// of its bitset); blocks <= 0: rows of 128 nodes over the whole lattice,
// threads outside the region return at once.
cudaError_t launch_lbm_near(const void *fin, void *fout, float4 *F, const LbmParams &p, const unsigned *bits,
                            float4 *vel, int blocks, const unsigned *seed, unsigned *next_seed, cudaStream_t s);
// Shared-memory opt-in of the list-form near field (its per-block running
// counts of the region bitset; once per context, before any capture).
cudaError_t prepare_near_field(long long max_words);
// True for the device functions of the far-field kernels (to tell their graph
// nodes apart).
bool is_lbm_far_kernel(const void *fn);
size_t pop_bytes(int fmt);
// K5: velocity u(t) (stored by the near-field stream-collide) interpolated at
// x + u_cur; u_next = u_cur + velocity. A vertex that moves one lattice
// spacing or more along an axis sets ERR_MOVED: the next step's force region
// (this step's support grown by one node) would no longer hold its support.
// With mark.bits not null the same threads add the force region of the new
// positions (the support of x + u_next grown by one node: the region of the
// step after next) to `mark`, cleared by the caller.
// form 0: eight threads per vertex (each a share of the support, the shares
// summed by shuffles); 1: one thread per vertex. Both sum the same partial
// sums in the same tree with every operation rounded explicitly: the same
// bits.
cudaError_t launch_interp_advect(const MeshView &m, const float4 *vel, const LbmParams &p, const float4 *u_cur,
                                 float4 *u_next, unsigned *err, cudaStream_t s, int block = 0,
                                 const RegionSlot &mark = RegionSlot{nullptr}, int form = 0);
// Compression between plates and the adjoint (csrc/adjoint.cu).
// out = J_el v at displacements u (vertex sums of the corner tangents; uses m.fc).
cudaError_t launch_force_jvp(const MeshView &m, const float4 *u, const float4 *v, float4 *out, unsigned *err,
                             cudaStream_t s);
// grad[3 c + (0, 1, 2)] += scale * lambda . df/d(mu, kappa, w) per cell (double).
cudaError_t launch_param_vjp(const MeshView &m, const float4 *u, const float4 *lam, double scale, double *grad,
                             cudaStream_t s);
cudaError_t launch_plate_step(const MeshView &m, const float4 *u_in, const float4 *v_in, const float4 *fel,
                              float4 *u_out, float4 *v_out, float dt, float c, float kp, const float *zlo,
                              const float *zhi, unsigned *err, cudaStream_t s);
cudaError_t launch_plate_force(const MeshView &m, const float4 *u, float kp, const float *zlo, const float *zhi,
                               double *out, cudaStream_t s);
cudaError_t launch_adj_seed(const MeshView &m, const float4 *u, float kp, const float *zlo, const float *zhi,
                            const double *dF, float4 *lam, cudaStream_t s);
cudaError_t launch_adj_m(int n, const float4 *ly, const float4 *lv, float dt, float4 *mvec, cudaStream_t s);
cudaError_t launch_adj_step(const MeshView &m, const float4 *u, const float4 *jv, const float4 *mvec, float4 *ly,
                            float4 *lv, float dt, float c, float kp, const float *zlo, const float *zhi,
                            cudaStream_t s);
cudaError_t launch_pack3(const double *in, int n, float4 *out, cudaStream_t s);

cudaError_t launch_lbm_init(void *f, const LbmParams &p, cudaStream_t s);
// rho and u(t) of every node after a step. u is u(t) as the near field
// stored it (vel) on the last step's force region (bits, in the tiling of
// p; null: no region), and from the populations and F elsewhere.
cudaError_t launch_lbm_macro(const void *f, const float4 *F, const LbmParams &p, const unsigned *bits,
                             const float4 *vel, double *rho, double *u, cudaStream_t s);

}  // namespace cf
