// Compression between plates and its adjoint (differentiation of the elastic
// forces with respect to positions and to the moduli).
//
// The paper compresses a cell between a resting plate and a moving one, with
// a repulsive force keeping vertices out of the plates (Sec. 4.2; the form of
// that force is in the supplement): here a one-sided harmonic penalty per
// vertex, f_z = k (z_lo - z)_+ - k (z - z_hi)_+, and quasi-static relaxation
// by damped steps of unit-mass vertices,
//   v <- c v + dt (f_el(y) + f_plate(y)),  y <- y + dt v   (0 <= c < 1;
// c = 0 is the first-order gradient flow y <- y + dt^2 f). The measured force
// is the top plate's, F = sum_v k (z_v - z_hi)_+.
//
// Adjoint of one step with (lambda_y, lambda_v) = dL/d(y, v) after it and
// m = dt lambda_y + lambda_v (the sensitivity to the new velocity):
//   lambda_y <- lambda_y + dt (J_el + J_plate) m,  lambda_v <- c m,
//   dL/dtheta += dt m . df/dtheta.
// J_el = -Hessian of the elastic energy is symmetric, so J_el m is the
// directional derivative of the forces along m: k_tet_jvp runs the force
// evaluation of mr.cuh on dual numbers. The forces are linear in
// (mu_1, mu_2, kappa), so m . df/d(mu, kappa, w) comes from the forces at unit
// moduli (k_param_vjp), reduced in double.
#include "mr.cuh"

namespace cf {

// ---------------------------------------------------------------- JVP
// Corner tangents d f / d eps of f(u + eps v) into m.fc.
__global__ void __launch_bounds__(128) k_tet_jvp(MeshView m, const float4 *__restrict__ u,
                                                 const float4 *__restrict__ v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const int4 a4 = __ldg(m.tet + t);
    float Bm[3][3];
    load_B(m, t, Bm);
    float H[3][3], dH[3][3];
    tet_grad(__ldg(u + a4.x), __ldg(u + a4.y), __ldg(u + a4.z), __ldg(u + a4.w), Bm, H);
    tet_grad(__ldg(v + a4.x), __ldg(v + a4.y), __ldg(v + a4.z), __ldg(v + a4.w), Bm, dH);
    Dual Hd[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Hd[i][j] = Dual(H[i][j], dH[i][j]);
    const float4 mat = __ldg(m.mat + mat_slot(m, t));
    InvT<Dual> inv;
    Dual P[3][3];
    mr_stress(Hd, mat.x, mat.y, mat.z, inv, P);
    float dP[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dP[i][j] = P[i][j].d;
    float f[4][3];
    corner_forces(dP, Bm, __ldg(m.V0 + t), f);
#pragma unroll
    for (int a = 0; a < 4; ++a) m.fc[a * m.T + t] = make_float4(f[a][0], f[a][1], f[a][2], 0.f);
}

cudaError_t launch_force_jvp(const MeshView &m, const float4 *u, const float4 *v, float4 *out, unsigned *err,
                             cudaStream_t s) {
    if (m.T == 0) return cudaSuccess;
    k_tet_jvp<<<(m.T + 127) / 128, 128, 0, s>>>(m, u, v);
    MeshView g = m;
    g.fv = out;
    return launch_gather_spread(g, u, nullptr, nullptr, err, s);
}

// ---------------------------------------------------------------- parameters
// Sum of `val` over the lanes of a warp that share cell c, added into
// dst[stride * c] once per warp when the whole warp has one cell (elements
// of a cell are contiguous, so that is the common case). Every lane calls;
// c < 0 marks lanes without an element.
__device__ __forceinline__ void warp_cell_add(int c, double val, double *dst, int stride) {
    const unsigned full = 0xffffffffu;
    const int c0 = __shfl_sync(full, c, 0);
    if (__all_sync(full, c == c0)) {
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(full, val, o);
        if ((threadIdx.x & 31) == 0 && c >= 0) atomicAdd(dst + stride * c, val);
    } else if (c >= 0) {
        atomicAdd(dst + stride * c, val);
    }
}

// lambda . df/d(mu, kappa, w) per cell, times `scale`, added into grad[3 c + .].
__global__ void __launch_bounds__(128) k_param_vjp(MeshView m, const float4 *__restrict__ u,
                                                   const float4 *__restrict__ lam, double scale, double *grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    double dmu = 0.0, dkappa = 0.0, dw = 0.0;
    if (t < m.T) {
        const int4 a4 = __ldg(m.tet + t);
        float Bm[3][3];
        load_B(m, t, Bm);
        float H[3][3];
        tet_grad(__ldg(u + a4.x), __ldg(u + a4.y), __ldg(u + a4.z), __ldg(u + a4.w), Bm, H);
        const float4 l[4] = {__ldg(lam + a4.x), __ldg(lam + a4.y), __ldg(lam + a4.z), __ldg(lam + a4.w)};
        const float V0 = __ldg(m.V0 + t);
        double g[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {  // unit mu1, unit mu2, unit kappa
            InvT<float> inv;
            float P[3][3], f[4][3];
            mr_stress(H, k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f, inv, P);
            corner_forces(P, Bm, V0, f);
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) s += (double)l[a].x * f[a][0] + (double)l[a].y * f[a][1] + (double)l[a].z * f[a][2];
            g[k] = s;
        }
        c = __ldg(m.tcell + t);
        const float4 mat = __ldg(m.mat + c);  // mu1, mu2, kappa, w
        const double mu = (double)mat.x + (double)mat.y, w = (double)mat.w;
        dmu = scale * (w * g[0] + (1.0 - w) * g[1]);
        dkappa = scale * g[2];
        dw = scale * mu * (g[0] - g[1]);
    }
    warp_cell_add(c, dmu, grad, 3);
    warp_cell_add(c, dkappa, grad + 1, 3);
    warp_cell_add(c, dw, grad + 2, 3);
}

cudaError_t launch_param_vjp(const MeshView &m, const float4 *u, const float4 *lam, double scale, double *grad,
                             cudaStream_t s) {
    if (m.T == 0) return cudaSuccess;
    k_param_vjp<<<(m.T + 127) / 128, 128, 0, s>>>(m, u, lam, scale, grad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- plates
struct PlateZ {
    float lo, hi;  // plate heights relative to the cell's integer origin
};

__device__ __forceinline__ PlateZ plates_of(const MeshView &m, int c, const float *zlo, const float *zhi) {
    const float oz = (float)__ldg(m.origin + 3 * c + 2);
    return {__ldg(zlo + c) - oz, __ldg(zhi + c) - oz};
}

// v <- c v + dt (f_el + f_plate), y <- y + dt v from (u_in, v_in) into
// (u_out, v_out); outputs may alias inputs.
__global__ void k_plate_step(MeshView m, const float4 *u_in, const float4 *v_in, const float4 *__restrict__ fel,
                             float4 *u_out, float4 *v_out, float dt, float c, float kp, const float *__restrict__ zlo,
                             const float *__restrict__ zhi, unsigned *err) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const float4 xr = __ldg(m.xr + v);
    const PlateZ pz = plates_of(m, __float_as_int(xr.w), zlo, zhi);
    const float4 uu = u_in[v], vv = v_in[v], f = fel[v];
    const float z = xr.z + uu.z;
    const float fz = f.z + kp * fmaxf(pz.lo - z, 0.f) - kp * fmaxf(z - pz.hi, 0.f);
    const float4 vn = make_float4(c * vv.x + dt * f.x, c * vv.y + dt * f.y, c * vv.z + dt * fz, 0.f);
    const float4 un = make_float4(uu.x + dt * vn.x, uu.y + dt * vn.y, uu.z + dt * vn.z, 0.f);
    if (!isfinite(un.x + un.y + un.z)) atomicOr(err, ERR_NONFINITE);
    u_out[v] = un;
    v_out[v] = vn;
}

cudaError_t launch_plate_step(const MeshView &m, const float4 *u_in, const float4 *v_in, const float4 *fel,
                              float4 *u_out, float4 *v_out, float dt, float c, float kp, const float *zlo,
                              const float *zhi, unsigned *err, cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    k_plate_step<<<(m.V + 255) / 256, 256, 0, s>>>(m, u_in, v_in, fel, u_out, v_out, dt, c, kp, zlo, zhi, err);
    return cudaGetLastError();
}

// F_c = sum over the cell's vertices of k (z - z_hi)_+ (added into out[c]).
__global__ void k_plate_force(MeshView m, const float4 *__restrict__ u, float kp, const float *__restrict__ zlo,
                              const float *__restrict__ zhi, double *out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    int c = -1;
    double f = 0.0;
    if (v < m.V) {
        const float4 xr = __ldg(m.xr + v);
        c = __float_as_int(xr.w);
        const PlateZ pz = plates_of(m, c, zlo, zhi);
        f = (double)kp * (double)fmaxf(xr.z + __ldg(u + v).z - pz.hi, 0.f);
    }
    warp_cell_add(c, f, out, 1);
}

cudaError_t launch_plate_force(const MeshView &m, const float4 *u, float kp, const float *zlo, const float *zhi,
                               double *out, cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    k_plate_force<<<(m.V + 255) / 256, 256, 0, s>>>(m, u, kp, zlo, zhi, out);
    return cudaGetLastError();
}

// lambda_z += dL/dF_c * dF_c/dz_v = dF[c] k [z_v > z_hi].
__global__ void k_adj_seed(MeshView m, const float4 *__restrict__ u, float kp, const float *__restrict__ zlo,
                           const float *__restrict__ zhi, const double *__restrict__ dF, float4 *lam) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const float4 xr = __ldg(m.xr + v);
    const int c = __float_as_int(xr.w);
    const PlateZ pz = plates_of(m, c, zlo, zhi);
    if (xr.z + __ldg(u + v).z > pz.hi) lam[v].z += (float)(__ldg(dF + c) * (double)kp);
}

// m = dt lambda_y + lambda_v
__global__ void k_adj_m(int n, const float4 *__restrict__ ly, const float4 *__restrict__ lv, float dt, float4 *mvec) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const float4 a = __ldg(ly + v), b = __ldg(lv + v);
    mvec[v] = make_float4(fmaf(dt, a.x, b.x), fmaf(dt, a.y, b.y), fmaf(dt, a.z, b.z), 0.f);
}

// lambda_y <- lambda_y + dt (J_el m + J_plate m), lambda_v <- c m at positions
// u, with J_el m given (jv) and J_plate = diag(0, 0, -k) on penetrating
// vertices.
__global__ void k_adj_step(MeshView m, const float4 *__restrict__ u, const float4 *__restrict__ jv,
                           const float4 *__restrict__ mvec, float4 *ly, float4 *lv, float dt, float c, float kp,
                           const float *__restrict__ zlo, const float *__restrict__ zhi) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const float4 xr = __ldg(m.xr + v);
    const PlateZ pz = plates_of(m, __float_as_int(xr.w), zlo, zhi);
    const float z = xr.z + __ldg(u + v).z;
    const float4 l = ly[v], j = __ldg(jv + v), mm = __ldg(mvec + v);
    const float jz = (z < pz.lo || z > pz.hi) ? -kp * mm.z : 0.f;
    ly[v] = make_float4(l.x + dt * j.x, l.y + dt * j.y, l.z + dt * (j.z + jz), 0.f);
    lv[v] = make_float4(c * mm.x, c * mm.y, c * mm.z, 0.f);
}

cudaError_t launch_adj_seed(const MeshView &m, const float4 *u, float kp, const float *zlo, const float *zhi,
                            const double *dF, float4 *lam, cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    k_adj_seed<<<(m.V + 255) / 256, 256, 0, s>>>(m, u, kp, zlo, zhi, dF, lam);
    return cudaGetLastError();
}

cudaError_t launch_adj_m(int n, const float4 *ly, const float4 *lv, float dt, float4 *mvec, cudaStream_t s) {
    if (n > 0) k_adj_m<<<(n + 255) / 256, 256, 0, s>>>(n, ly, lv, dt, mvec);
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const MeshView &m, const float4 *u, const float4 *jv, const float4 *mvec, float4 *ly,
                            float4 *lv, float dt, float c, float kp, const float *zlo, const float *zhi,
                            cudaStream_t s) {
    if (m.V == 0) return cudaSuccess;
    k_adj_step<<<(m.V + 255) / 256, 256, 0, s>>>(m, u, jv, mvec, ly, lv, dt, c, kp, zlo, zhi);
    return cudaGetLastError();
}

// double [n][3] (host layout) -> float4 [n]
__global__ void k_pack3(const double *__restrict__ in, int n, float4 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4((float)in[3 * i], (float)in[3 * i + 1], (float)in[3 * i + 2], 0.f);
}

cudaError_t launch_pack3(const double *in, int n, float4 *out, cudaStream_t s) {
    if (n > 0) k_pack3<<<(n + 255) / 256, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

}  // namespace cf
