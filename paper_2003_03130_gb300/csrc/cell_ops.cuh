// Per-element bodies of the cell kernels, shared by the separate launches
// (csrc/tet_force.cu, csrc/ibm.cu) and the fused persistent chain
// (csrc/chain.cu): tet corner forces, the per-vertex region marking, the
// vertex sum with its spread, and the interpolation's partial sums.
#pragma once

#include "mr.cuh"

namespace cf {

// Everything the force of one tet reads: its four displacements, B, V0 and
// its material.
struct TetIn {
    float4 w[4];
    float Bm[3][3];
    float V0;
    float4 mat;
};

__device__ __forceinline__ void tet_load(const MeshView &m, const float4 *__restrict__ u, int t, TetIn &in) {
    const int4 a4 = __ldg(m.tet + t);
    int slot;
    load_tet_params(m, t, in.Bm, in.V0, slot);
    in.w[0] = __ldg(u + a4.x);
    in.w[1] = __ldg(u + a4.y);
    in.w[2] = __ldg(u + a4.z);
    in.w[3] = __ldg(u + a4.w);
    in.mat = __ldg(m.mat + slot);
}

// Corner forces of tet t from its inputs (Sec. 3.1): f^a = -V0 P B_a,
// f^4 = -(f^1 + f^2 + f^3).
__device__ __forceinline__ void tet_forces_store(const MeshView &m, const TetIn &in, unsigned *err, int t) {
    float H[3][3];
    tet_grad(in.w[0], in.w[1], in.w[2], in.w[3], in.Bm, H);
    InvT<float> v;
    float P[3][3];
    invariants_t(H, v);
    if (needs_fp64_volume(m, in.mat))
        set_volume_change(v, (float)volume_change64(m.B64, m.T, t, in.w[0], in.w[1], in.w[2], in.w[3]));
    mr_stress_inv(H, in.mat.x, in.mat.y, in.mat.z, v, P);
    if (!(v.J > 0.f)) atomicOr(err, ERR_INVERTED);
    float f[4][3];
    corner_forces(P, in.Bm, in.V0, f);
#pragma unroll
    for (int a = 0; a < 4; ++a) m.fc[a * m.T + t] = make_float4(f[a][0], f[a][1], f[a][2], 0.f);
}

__device__ __forceinline__ void tet_corner_forces(const MeshView &m, const float4 *__restrict__ u, unsigned *err,
                                                  int t) {
    TetIn in;
    tet_load(m, u, t, in);
    tet_forces_store(m, in, err, t);
}

// The per-vertex part of K1 when it marks the region: add the next step's
// force region (the support of x + u grown by one node) to mark. Whether this
// step's support lies in this step's region follows from the step before
// moving every vertex by less than one spacing, which K5 checks.
template <int W>
__device__ __forceinline__ void mark_vertex(const MeshView &m, const float4 *__restrict__ u, const LbmParams &lp,
                                            int v, const RegionSlot &mark) {
    Support s;
    if (support_of<W>(m.origin, __ldg(m.xr + v), __ldg(u + v), lp.ny, s))  // else K23 reports it
        mark_region<W>(s, lp, mark);
}

// ---- K5 in a fixed rounding order
// The interpolation of u(t) at a vertex is split into eight partial sums:
// for W = 2 partial k is the corner (dx, dy, dz) = (k & 1, (k >> 1) & 1,
// k >> 2), for W = 4 the plane dz = k >> 1, rows dy = 2 (k & 1) + {0, 1},
// x fastest. They meet in the tree ((p0 + p1) + (p2 + p3)) + ((p4 + p5) +
// (p6 + p7)). Every product and sum is rounded explicitly (no contraction),
// so the eight-thread form (one partial per thread, the tree by xor
// shuffles) and the one-thread form give the same bits.
__device__ __forceinline__ float3 add3_rn(float3 a, float3 b) {
    return make_float3(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z));
}

template <int W>
__device__ __forceinline__ float3 interp_partial(const Support &s, const float (&wx)[W], const float (&wy)[W],
                                                 const float (&wz)[W], const float4 *__restrict__ vel,
                                                 const LbmParams &p, int k) {
    if constexpr (W == 2) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
        const int n = wrapi(s.bx + dx, p.nx) + p.nx * (s.by + dy + p.ny * wrapi(s.bz + dz, p.nz));
        const float w = __fmul_rn(__fmul_rn(wx[dx], wy[dy]), wz[dz]);
        const float4 q = __ldg(vel + n);
        return make_float3(__fmul_rn(w, q.x), __fmul_rn(w, q.y), __fmul_rn(w, q.z));
    } else {
        const int dz = k >> 1, dy0 = 2 * (k & 1);
        const int Z = wrapi(s.bz + dz, p.nz);
        float3 a = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int dy = dy0 + j;
            const int row = p.nx * (s.by + dy + p.ny * Z);
            const float wyz = __fmul_rn(wy[dy], wz[dz]);
#pragma unroll
            for (int dx = 0; dx < W; ++dx) {
                const float w = __fmul_rn(wx[dx], wyz);
                const float4 q = __ldg(vel + wrapi(s.bx + dx, p.nx) + row);
                a.x = __fmaf_rn(w, q.x, a.x);
                a.y = __fmaf_rn(w, q.y, a.y);
                a.z = __fmaf_rn(w, q.z, a.z);
            }
        }
        return a;
    }
}

// The interpolated u(t) at x + u_cur (d) in one thread; false if that
// position's support is not valid.
template <int W>
__device__ __forceinline__ bool interp_vertex(const MeshView &m, const float4 *__restrict__ vel, const LbmParams &p,
                                              float4 xr, float4 uc, Support &s, float3 &d) {
    d = make_float3(0.f, 0.f, 0.f);
    if (!support_of<W>(m.origin, xr, uc, p.ny, s)) return false;
    float wx[W], wy[W], wz[W];
    delta_weights<W>(s.fx, wx);
    delta_weights<W>(s.fy, wy);
    delta_weights<W>(s.fz, wz);
    float3 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = interp_partial<W>(s, wx, wy, wz, vel, p, k);
    d = add3_rn(add3_rn(add3_rn(a[0], a[1]), add3_rn(a[2], a[3])), add3_rn(add3_rn(a[4], a[5]), add3_rn(a[6], a[7])));
    return true;
}

// Corner-force load: from L2 (FC_L2) when the forces were written by other
// blocks of the same launch, so that no stale L1 line is read.
template <bool FC_L2>
__device__ __forceinline__ float4 load_fc(const float4 *p) {
    if constexpr (FC_L2)
        return __ldcg(p);
    else
        return *p;
}

// Vertex force of vertex v by four lanes (lane 0..3; every lane of the warp
// takes part in the shuffles, `live` false for padding lanes): lane k sums
// the entries k, k+4, k+8, ... of the incidence row, and the four partial
// sums are combined by a fixed shuffle tree (the same order every call:
// deterministic). Every lane of the group ends with the sum.
template <bool FC_L2>
__device__ __forceinline__ void gather_vertex(const MeshView &m, int v, int lane, bool live, float &fx, float &fy,
                                              float &fz) {
    fx = fy = fz = 0.f;
    if (live) {
        // the lane's entries e0 + lane, + 4, + 8, ... in groups of four: the
        // index loads of a group, then its corner-force loads, are issued
        // together; the sum still runs over the entries in ascending order
        const int e0 = __ldg(m.csr_ptr + v), e1 = __ldg(m.csr_ptr + v + 1);
        for (int e = e0 + lane; e < e1; e += 16) {
            int id[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) id[k] = e + 4 * k < e1 ? __ldg(m.csr_idx + e + 4 * k) : -1;
            float4 c[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                c[k] = id[k] >= 0 ? load_fc<FC_L2>(m.fc + (id[k] & 3) * m.T + (id[k] >> 2)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (id[k] >= 0) {
                    fx += c[k].x;
                    fy += c[k].y;
                    fz += c[k].z;
                }
        }
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
}

// The spread of one vertex's force (fx, fy, fz) onto its support s, lane
// `lane` of four taking its share of the support nodes: for W = 2 lane
// (dz, dy) the two nodes of its x row, for W = 4 lane dz the W x W plane.
// sink(X, Y, Z, w) receives each node with x and z not yet wrapped and its
// weight w.
template <int W, class Sink>
__device__ __forceinline__ void spread_vertex(const Support &s, int lane, Sink &&sink) {
    float wx[W], wy[W], wz[W];
    delta_weights<W>(s.fx, wx);
    delta_weights<W>(s.fy, wy);
    delta_weights<W>(s.fz, wz);
    if constexpr (W == 2) {
        const int dz = lane >> 1, dy = lane & 1;
        const float wyz = wy[dy] * wz[dz];
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) sink(s.bx + dx, s.by + dy, s.bz + dz, wx[dx] * wyz);
    } else {
        float wzl = wz[0];
#pragma unroll
        for (int k = 1; k < W; ++k) wzl = lane == k ? wz[k] : wzl;  // no local-memory indexing
#pragma unroll
        for (int dy = 0; dy < W; ++dy) {
            const float wyz = wy[dy] * wzl;
#pragma unroll
            for (int dx = 0; dx < W; ++dx) sink(s.bx + dx, s.by + dy, s.bz + lane, wx[dx] * wyz);
        }
    }
}

// Vertex force of vertex v (four lanes, see gather_vertex) and, with
// do_spread, its spread onto F with one atomic per support node (one float4
// reduction, or three fixed-point ones with the deterministic spread).
template <int W, bool FC_L2>
__device__ __forceinline__ void gather_spread_vertex(const MeshView &m, const float4 *__restrict__ u, float4 *F,
                                                     const LbmParams &p, int do_spread, unsigned *err, int v,
                                                     int lane, bool live) {
    float fx, fy, fz;
    gather_vertex<FC_L2>(m, v, lane, live, fx, fy, fz);
    if (!live) return;
    if (lane == 0) {
        m.fv[v] = make_float4(fx, fy, fz, 0.f);
        if (!isfinite(fx + fy + fz)) atomicOr(err, ERR_NONFINITE);
    }
    if (!do_spread) return;
    Support s;
    if (!support_of<W>(m.origin, __ldg(m.xr + v), __ldg(u + v), p.ny, s)) {
        if (lane == 0) atomicOr(err, ERR_DOMAIN);
        return;
    }
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    spread_vertex<W>(s, lane, [&](int X, int Y, int Z, float w) {
        const int n = wrapi(X, nx) + nx * (Y + ny * wrapi(Z, nz));
        force_add(F, p, n, w * fx, w * fy, w * fz);
    });
}

}  // namespace cf
