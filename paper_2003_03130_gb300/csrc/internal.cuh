// Internal declarations of the GB300 cell/fluid library: device layouts,
// kernel launchers and the D3Q19 lattice as compile-time constants.
//
// Device layout (structure of arrays throughout, so that consecutive threads
// touch consecutive words):
//   populations  f[q * N + n], q = 0..18, n = x + nx*(y + ny*z), stored as the
//                deviation f_q - w_q from the rest equilibrium (keeps FP32
//                rounding relative to the O(u) signal, not to O(w_q));
//   force field  F[a * N + n], a = 0..2;
//   vertices     float4 per vertex (one 16-byte load in the tet gathers):
//                xr (FP32 x_ref relative to the cell's integer origin, .w =
//                cell id), u (FP32 displacement y - x_ref), fv (force);
//                xref64 [V][3] FP64 for exact host round trips;
//   tets         int4 tet[t], B[(3k + j) * T + t], V0[t], tcell[t];
//   corner force float4 fc[c * T + t].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cf {

// Error bits of the device error word (never trapped; read by the host).
enum : unsigned {
    ERR_INVERTED = 1u << 0,   // det F <= 0 in some tet
    ERR_NONFINITE = 1u << 1,  // NaN / Inf in a force or a displacement
    ERR_DOMAIN = 1u << 2,     // delta support outside 0 <= y <= ny-1
    ERR_MOVED = 1u << 3,      // a support node fell outside the step's force region
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
    int nx, ny, nz;
    long long N;
    float omega;        // 1/tau
    float guo;          // 1 - 1/(2 tau)
    float uw_lo, uw_hi; // wall x velocities at y = -1/2 and y = ny - 1/2
    float gx, gy, gz;   // uniform body-force density
    int dw;             // delta kernel: support width 2 (trilinear) or 4 (Peskin)
};

struct MeshView {
    int V, T;
    const float4 *xr;      // [V]: x_ref - origin (FP32), .w = cell id (int bits)
    const int *origin;     // [3 * ncells], integer origin of each cell
    const int4 *tet;       // [T]: global vertex indices, corner 3 = vertex 4
    const float *B;        // [9][T]: B[(3k + j) * T + t] = (J^-1)_kj
    const float *V0;       // [T]
    const int *tcell;      // [T]
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
// and the clearing of F so that all three see exactly the same node set.
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
template <>
__device__ __forceinline__ void delta_weights<4>(float f, float (&w)[4]) {
    const float q = sqrtf(fmaf(4.f * f, 1.f - f, 1.f));
    w[0] = 0.125f * (3.f - 2.f * f - q);
    w[1] = 0.125f * (3.f - 2.f * f + q);
    w[2] = 0.125f * (1.f + 2.f * f + q);
    w[3] = 0.125f * (1.f + 2.f * f - q);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Force region of a step. A box slot holds the bounding box of the delta
// support nodes of all vertices as 6 ints {min x, min y, min z, -max x,
// -max y, -max z} (x and z wrapped into the lattice), all accumulated with
// atomicMin from INT_MAX. The region a step uses is that box grown by one
// node in every direction (x, z periodic as start + length; y clamped).
struct NodeBox {
    int x0, lx, y0, y1, z0, lz;
};

__device__ __forceinline__ NodeBox region_of(const int *__restrict__ slot, int nx, int ny, int nz) {
    NodeBox b;
    const int xmin = slot[0], ymin = slot[1], zmin = slot[2];
    const int xmax = -slot[3], ymax = -slot[4], zmax = -slot[5];
    if (xmin > xmax) {  // empty: no vertex spread anything
        b.x0 = 0; b.lx = 0; b.y0 = 1; b.y1 = 0; b.z0 = 0; b.lz = 0;
        return b;
    }
    b.lx = xmax - xmin + 3;
    b.x0 = xmin - 1;
    if (b.lx >= nx) { b.x0 = 0; b.lx = nx; }
    b.lz = zmax - zmin + 3;
    b.z0 = zmin - 1;
    if (b.lz >= nz) { b.z0 = 0; b.lz = nz; }
    b.y0 = ymin - 1 < 0 ? 0 : ymin - 1;
    b.y1 = ymax + 1 > ny - 1 ? ny - 1 : ymax + 1;
    return b;
}

// offset of a periodic coordinate from the region start, in [0, n)
__device__ __forceinline__ int region_off(int c, int c0, int n) {
    int d = c - c0;
    d %= n;
    return d < 0 ? d + n : d;
}

__device__ __forceinline__ bool in_region(const NodeBox &b, int x, int y, int z, int nx, int nz) {
    return y >= b.y0 && y <= b.y1 && region_off(x, b.x0, nx) < b.lx && region_off(z, b.z0, nz) < b.lz;
}

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return the launch status.
// Once per cell (Sec. 3.2): validate, orient, B = J^-1 and V_0 in FP64;
// *status receives min over failing tets of ((t_report + t) << 8 | code),
// code 1 = index out of range, 2 = repeated vertex, 3 = degenerate.
cudaError_t launch_mesh_prepare(const double *x64, int nv, const int *tets_in, int nt, int v_off, int t_off,
                                int t_report, int T, int cell, int4 *tet, float *B, float *V0, int *tcell,
                                unsigned long long *status, cudaStream_t s);
cudaError_t launch_vertex_prepare(const double *x64, const double *y64, int nv, int v_off, int cell,
                                  const int *origin_host3, float4 *xr, float4 *u0, float4 *u1, double *xref64,
                                  cudaStream_t s);
cudaError_t launch_csr_build(const int4 *tet, int T, int V, int *ptr, int *idx, int *cursor, cudaStream_t s);
cudaError_t launch_set_positions(const double *y64, int v0, int nv, const double *xref64, float4 *u,
                                 cudaStream_t s);
cudaError_t launch_get_positions(const float4 *u, const double *xref64, int v0, int nv, double *y64,
                                 cudaStream_t s);
cudaError_t launch_get_forces(const float4 *fv, int v0, int nv, double *out, cudaStream_t s);

// K1: elastic corner forces of all tets at displacements u; when `u_prev` is
// non-null the same launch also zeroes the force field on the delta support
// of the positions x + u_prev (where the previous step spread its forces).
cudaError_t launch_tet_force(const MeshView &m, const float4 *u, unsigned *err, const float4 *u_prev, float *F,
                             const LbmParams *lp, cudaStream_t s);
// Per-tet V_0 U of tets [t0, t1) reduced in a fixed order into *out (double).
cudaError_t launch_energy(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s);
// K8: Taylor deformation of tets [t0, t1) at displacements u; out[10] (device)
// = D, D from the printed squared expression, inclination (deg), a1, a2, a3,
// theta1, theta2, theta3, volume. partial: 10 doubles per 256 tets.
cudaError_t launch_taylor(const MeshView &m, const float4 *u, int t0, int t1, double *partial, double *out,
                          cudaStream_t s);
// K2 (+K3): vertex force sums over the incidence rows; with F != null the
// same threads spread their vertex force onto the lattice. With box_out the
// bounding box of the support nodes is accumulated into that slot; with
// box_in every support node must lie in the region of that slot (else
// ERR_MOVED).
cudaError_t launch_gather_spread(const MeshView &m, const float4 *u, float *F, const LbmParams *lp, unsigned *err,
                                 cudaStream_t s, int *box_out = nullptr, const int *box_in = nullptr);
// Bounding box of the support nodes of x + u into a slot (reset by the caller).
cudaError_t launch_support_box(const MeshView &m, const float4 *u, const LbmParams &p, int *box_out,
                               cudaStream_t s);
// K4: pull stream + BGK collide with Guo forcing, fin -> fout, every node, no
// force field (fluid-only runs). Population buffers are in the format p.fmt.
cudaError_t launch_lbm(const void *fin, void *fout, const LbmParams &p, cudaStream_t s);
// K4 split by the force region of a slot: far = every node outside it, with
// no force-field read; near = the nodes inside it, with the force field, also
// storing u(t) there.
cudaError_t launch_lbm_far(const void *fin, void *fout, const LbmParams &p, const int *box, cudaStream_t s);
cudaError_t launch_lbm_near(const void *fin, void *fout, const float *F, const LbmParams &p, const int *box,
                            float *vel, cudaStream_t s);
// True for the device functions of the far-field kernels (to tell their graph
// nodes apart).
bool is_lbm_far_kernel(const void *fn);
size_t pop_bytes(int fmt);
// K5: velocity u(t) (stored by the near-field stream-collide) interpolated at
// x + u_cur; u_next = u_cur + velocity.
cudaError_t launch_interp_advect(const MeshView &m, const float *vel, const LbmParams &p, const float4 *u_cur,
                                 float4 *u_next, unsigned *err, cudaStream_t s);
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
cudaError_t launch_lbm_macro(const void *f, const float *F, const LbmParams &p, double *rho, double *u,
                             cudaStream_t s);

}  // namespace cf
