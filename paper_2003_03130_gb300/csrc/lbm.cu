// K4: D3Q19 lattice-Boltzmann stream + collide (the fluid of Sec. 6; the
// paper uses ESPResSo's LB without stating the operator). One thread per
// node, pull scheme: the buffer holds post-collision populations, a node
// pulls f_q(x - c_q) from the old buffer, collides, and writes the new
// post-collision populations at x into the other buffer. Populations are
// stored as deviations d_q = f_q - w_q, so rest equilibrium is all zeros and
// every FP32 operation is relative to the O(u) signal.
//
//   walls (Sec. 6.1 moving planes): a pull from beyond y = -1/2 or
//     y = ny - 1/2 is halfway bounce-back with the moving-wall term,
//     f_q(x) = f*_opp(q)(x) + 6 w_q (c_q . u_wall)  (rho_0 = 1);
//   moments: rho = 1 + sum d_q, rho u = sum c_q d_q + F/2, F = F(x) + g;
//   BGK + Guo: d*_q = d_q + omega (d^eq_q - d_q)
//                     + (1 - omega/2) w_q [3 (c_q - u) + 9 (c_q . u) c_q] . F,
//     d^eq_q = w_q [(rho - 1) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)].
// Loads along x are coalesced (scalar, unit stride, possibly shifted by one
// word); stores are unit-stride.
#include "internal.cuh"

namespace cf {

template <bool HAS_F>
__global__ void __launch_bounds__(128) k_lbm(const float *__restrict__ fin, float *__restrict__ fout,
                                             const float *__restrict__ F, LbmParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int N = (int)p.N;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int n = x + nx * (y + ny * z);

    float d[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : x);
        const int sy = y - cy(q);
        const int sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z);
        if (cy(q) != 0 && (sy < 0 || sy >= ny)) {
            const float uw = sy < 0 ? p.uw_lo : p.uw_hi;
            d[q] = __ldg(fin + opp(q) * N + n) + (6.f * wq(q) * cx(q)) * uw;
        } else {
            d[q] = __ldg(fin + q * N + sx + nx * (sy + ny * sz));
        }
    }

    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += d[q];
        if (cx(q)) jx += cx(q) * d[q];
        if (cy(q)) jy += cy(q) * d[q];
        if (cz(q)) jz += cz(q) * d[q];
    }
    float Fx = p.gx, Fy = p.gy, Fz = p.gz;
    if (HAS_F) {
        Fx += __ldg(F + n);
        Fy += __ldg(F + N + n);
        Fz += __ldg(F + 2 * N + n);
    }
    const float rho = 1.f + drho;
    const float ir = 1.f / rho;
    const float ux = (jx + 0.5f * Fx) * ir, uy = (jy + 0.5f * Fy) * ir, uz = (jz + 0.5f * Fz) * ir;
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    const float om = p.omega, g = p.guo;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
        const float cF = cx(q) * Fx + cy(q) * Fy + cz(q) * Fz;
        const float deq = wq(q) * (drho + rho * (3.f * cu + 4.5f * cu * cu - usq));
        const float src = (g * wq(q)) * (3.f * (cF - uF) + 9.f * cu * cF);
        fout[q * N + n] = d[q] + om * (deq - d[q]) + src;
    }
}

cudaError_t launch_lbm(const float *fin, float *fout, const float *F, const LbmParams &p, cudaStream_t s) {
    const int bx = p.nx < 128 ? p.nx : 128;
    dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
    if (F)
        k_lbm<true><<<grid, bx, 0, s>>>(fin, fout, F, p);
    else
        k_lbm<false><<<grid, bx, 0, s>>>(fin, fout, F, p);
    return cudaGetLastError();
}

cudaError_t launch_lbm_init(float *f, const LbmParams &p, cudaStream_t s) {
    // rest equilibrium, rho = 1, u = 0: every deviation is zero
    return cudaMemsetAsync(f, 0, sizeof(float) * 19 * (size_t)p.N, s);
}

// rho and u(t) on every node from post-collision populations and the force of
// the same step: rho = 1 + sum d*_q, rho u = sum c_q d*_q - F/2.
__global__ void k_macro(const float *__restrict__ f, const float *__restrict__ F, LbmParams p, double *rho,
                        double *u) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = (int)p.N;
    if (n >= N) return;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float d = f[q * N + n];
        drho += d;
        if (cx(q)) jx += cx(q) * d;
        if (cy(q)) jy += cy(q) * d;
        if (cz(q)) jz += cz(q) * d;
    }
    const float Fx = F[n] + p.gx, Fy = F[N + n] + p.gy, Fz = F[2 * N + n] + p.gz;
    const float r = 1.f + drho;
    if (rho) rho[n] = (double)r;
    if (u) {
        u[3 * (size_t)n + 0] = (double)((jx - 0.5f * Fx) / r);
        u[3 * (size_t)n + 1] = (double)((jy - 0.5f * Fy) / r);
        u[3 * (size_t)n + 2] = (double)((jz - 0.5f * Fz) / r);
    }
}

cudaError_t launch_lbm_macro(const float *f, const float *F, const LbmParams &p, double *rho, double *u,
                             cudaStream_t s) {
    k_macro<<<(int)((p.N + 255) / 256), 256, 0, s>>>(f, F, p, rho, u);
    return cudaGetLastError();
}

}  // namespace cf
