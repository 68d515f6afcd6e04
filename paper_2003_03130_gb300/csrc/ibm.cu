// Immersed-boundary coupling (Sec. 6: the cell is coupled to the fluid by an
// immersed-boundary method; the kernel is not given there). Trilinear
// two-point delta: delta_h(r) = phi(r_x) phi(r_y) phi(r_z), phi(r) =
// max(0, 1 - |r|), nonzero on the 8 nodes floor(y) + {0,1}^3. Every vertex,
// interior ones included, is a coupling point (the fluid fills the cell).
//
// K2+K3 (k_gather_spread), one thread per vertex:
//   f_v = sum of the corner forces in the vertex's incidence row, in the
//         row's fixed ascending (tet, corner) order - deterministic, no
//         atomics (Sec. 3.1 defines forces per tet corner; the vertex force
//         is their sum);
//   F(x) += f_v delta_h(x - y_v) on the 8 support nodes (float atomics:
//         the spread field is exact up to the order of those additions).
// K5 (k_interp_advect), one thread per vertex:
//   u(t) on each support node from the post-collision populations through
//   rho u = sum_q c_q f*_q - F/2 (the collision adds exactly F to the
//   momentum, and rho u = sum_q c_q f_q + F/2 before it), then
//   y^{t+1} = y^t + sum_x u(x) delta_h(x - y^t).
#include "internal.cuh"

namespace cf {

__global__ void __launch_bounds__(256) k_gather_spread(MeshView m, const float4 *__restrict__ u, float *F, LbmParams p,
                                                       int do_spread, unsigned *err) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const int e0 = __ldg(m.csr_ptr + v), e1 = __ldg(m.csr_ptr + v + 1);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int e = e0; e < e1; ++e) {
        const int id = __ldg(m.csr_idx + e);
        const float4 c = m.fc[(id & 3) * m.T + (id >> 2)];
        fx += c.x;
        fy += c.y;
        fz += c.z;
    }
    m.fv[v] = make_float4(fx, fy, fz, 0.f);
    if (!isfinite(fx + fy + fz)) atomicOr(err, ERR_NONFINITE);
    if (!do_spread) return;
    Support s;
    if (!support_of(m.origin, __ldg(m.xr + v), __ldg(u + v), p.ny, s)) {
        atomicOr(err, ERR_DOMAIN);
        return;
    }
    const int N = (int)p.N;
    const float wx[2] = {1.f - s.fx, s.fx}, wy[2] = {1.f - s.fy, s.fy}, wz[2] = {1.f - s.fz, s.fz};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int Z = wrapi(s.bz + dz, p.nz);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int n = wrapi(s.bx + dx, p.nx) + p.nx * (s.by + dy + p.ny * Z);
                const float w = wx[dx] * wy[dy] * wz[dz];
                atomicAdd(F + n, w * fx);
                atomicAdd(F + N + n, w * fy);
                atomicAdd(F + 2 * N + n, w * fz);
            }
    }
}

cudaError_t launch_gather_spread(const MeshView &m, const float4 *u, float *F, const LbmParams *lp, unsigned *err,
                                 cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    LbmParams p{};
    if (lp) p = *lp;
    k_gather_spread<<<(m.V + 255) / 256, 256, 0, s>>>(m, u, F, p, (F && lp) ? 1 : 0, err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128) k_interp_advect(MeshView m, const float *__restrict__ f,
                                                       const float *__restrict__ F, LbmParams p,
                                                       const float4 *__restrict__ u_cur, float4 *u_next,
                                                       unsigned *err) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const float4 uc = __ldg(u_cur + v);
    Support s;
    if (!support_of(m.origin, __ldg(m.xr + v), uc, p.ny, s)) {
        atomicOr(err, ERR_DOMAIN);
        u_next[v] = uc;
        return;
    }
    const int N = (int)p.N;
    const float wx[2] = {1.f - s.fx, s.fx}, wy[2] = {1.f - s.fy, s.fy}, wz[2] = {1.f - s.fz, s.fz};
    float vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int Z = wrapi(s.bz + dz, p.nz);
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int n = wrapi(s.bx + dx, p.nx) + p.nx * (s.by + dy + p.ny * Z);
                float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                for (int q = 0; q < 19; ++q) {
                    const float d = __ldg(f + q * N + n);
                    drho += d;
                    if (cx(q)) jx += cx(q) * d;
                    if (cy(q)) jy += cy(q) * d;
                    if (cz(q)) jz += cz(q) * d;
                }
                const float Fx = __ldg(F + n) + p.gx, Fy = __ldg(F + N + n) + p.gy, Fz = __ldg(F + 2 * N + n) + p.gz;
                const float ir = 1.f / (1.f + drho);
                const float w = wx[dx] * wy[dy] * wz[dz];
                vx += w * ((jx - 0.5f * Fx) * ir);
                vy += w * ((jy - 0.5f * Fy) * ir);
                vz += w * ((jz - 0.5f * Fz) * ir);
            }
    }
    const float4 un = make_float4(uc.x + vx, uc.y + vy, uc.z + vz, 0.f);
    if (!isfinite(un.x + un.y + un.z)) atomicOr(err, ERR_NONFINITE);
    u_next[v] = un;
}

cudaError_t launch_interp_advect(const MeshView &m, const float *f, const float *F, const LbmParams &p,
                                 const float4 *u_cur, float4 *u_next, unsigned *err, cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    k_interp_advect<<<(m.V + 127) / 128, 128, 0, s>>>(m, f, F, p, u_cur, u_next, err);
    return cudaGetLastError();
}

}  // namespace cf
