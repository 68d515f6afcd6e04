// Once-per-cell set-up (Sec. 3.2: J and B = J^-1 depend only on the
// reference coordinates and are computed once), vertex incidence rows for the
// deterministic vertex-force sum, and host <-> device conversions of
// positions and forces. The precompute runs in FP64 on the device and stores
// FP32 (B also in FP64, for the volume term of nearly incompressible tets).
#include "internal.cuh"

namespace cf {

// One thread per tet of the new cell.
__global__ void k_mesh_prepare(const double *__restrict__ x64, int nv, const int *__restrict__ tets_in, int nt,
                               int v_off, int t_off, int t_report, int T, int cell, int4 *tet, float *B,
                               double *B64, float *V0, int *tcell, unsigned long long *status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int a[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) a[c] = tets_in[4 * t + c];
    unsigned code = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (a[c] < 0 || a[c] >= nv) code = 1;
    if (!code)
        for (int c = 0; c < 4; ++c)
            for (int e = c + 1; e < 4; ++e)
                if (a[c] == a[e]) code = 2;
    if (code) {
        atomicMin(status, ((unsigned long long)(t_report + t) << 8) | code);
        return;
    }
    double Jm[3][3];  // J_ik = x_i^k - x_i^4
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) Jm[i][k] = x64[3 * a[k] + i] - x64[3 * a[3] + i];
    double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                 Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                 Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
    double l2 = 0.0;
    for (int c = 0; c < 4; ++c)
        for (int e = c + 1; e < 4; ++e) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) {
                const double q = x64[3 * a[c] + i] - x64[3 * a[e] + i];
                s += q * q;
            }
            l2 = s > l2 ? s : l2;
        }
    const double lmax = sqrt(l2);
    if (fabs(det) <= 1e-12 * lmax * lmax * lmax) {
        atomicMin(status, ((unsigned long long)(t_report + t) << 8) | 3u);
        return;
    }
    if (det < 0.0) {  // swap corners 1 and 2: positively oriented
        const int s = a[0];
        a[0] = a[1];
        a[1] = s;
        for (int i = 0; i < 3; ++i) {
            const double q = Jm[i][0];
            Jm[i][0] = Jm[i][1];
            Jm[i][1] = q;
        }
        det = -det;
    }
    // B = J^-1 = adj(J) / det
    double Bi[3][3];
    Bi[0][0] = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
    Bi[0][1] = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
    Bi[0][2] = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
    Bi[1][0] = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
    Bi[1][1] = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
    Bi[1][2] = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
    Bi[2][0] = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
    Bi[2][1] = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
    Bi[2][2] = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
    const int tg = t_off + t;
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) {
            const double b = Bi[k][j] / det;
            B[(3 * k + j) * T + tg] = (float)b;
            B64[(3 * k + j) * T + tg] = b;
        }
    V0[tg] = (float)(det / 6.0);
    tet[tg] = make_int4(a[0] + v_off, a[1] + v_off, a[2] + v_off, a[3] + v_off);
    tcell[tg] = cell;
}

cudaError_t launch_mesh_prepare(const double *x64, int nv, const int *tets_in, int nt, int v_off, int t_off,
                                int t_report, int T, int cell, int4 *tet, float *B, double *B64, float *V0,
                                int *tcell, unsigned long long *status, cudaStream_t s) {
    k_mesh_prepare<<<(nt + 127) / 128, 128, 0, s>>>(x64, nv, tets_in, nt, v_off, t_off, t_report, T, cell, tet, B,
                                                    B64, V0, tcell, status);
    return cudaGetLastError();
}

// One thread per vertex of the new cell: FP32 reference position relative to
// the integer origin (cell id in .w), FP32 displacement, FP64 reference copy.
__global__ void k_vertex_prepare(const double *__restrict__ x64, const double *__restrict__ y64, int nv, int v_off,
                                 int cell, int ox, int oy, int oz, float4 *xr, float4 *u0, float4 *u1,
                                 double *xref64) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const double x = x64[3 * v], y = x64[3 * v + 1], z = x64[3 * v + 2];
    const double *yy = y64 ? y64 + 3 * v : x64 + 3 * v;
    const int g = v_off + v;
    xr[g] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), __int_as_float(cell));
    const float4 du = make_float4((float)(yy[0] - x), (float)(yy[1] - y), (float)(yy[2] - z), 0.f);
    u0[g] = du;
    u1[g] = du;
    xref64[3 * g] = x;
    xref64[3 * g + 1] = y;
    xref64[3 * g + 2] = z;
}

cudaError_t launch_vertex_prepare(const double *x64, const double *y64, int nv, int v_off, int cell,
                                  const int *origin_host3, float4 *xr, float4 *u0, float4 *u1, double *xref64,
                                  cudaStream_t s) {
    k_vertex_prepare<<<(nv + 127) / 128, 128, 0, s>>>(x64, y64, nv, v_off, cell, origin_host3[0], origin_host3[1],
                                                      origin_host3[2], xr, u0, u1, xref64);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- incidence
__global__ void k_csr_count(const int4 *__restrict__ tet, int T, int *cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int4 a = tet[t];
    atomicAdd(cnt + a.x + 1, 1);
    atomicAdd(cnt + a.y + 1, 1);
    atomicAdd(cnt + a.z + 1, 1);
    atomicAdd(cnt + a.w + 1, 1);
}

// Inclusive scan of ptr[1..V] in place by one block (set-up only).
__global__ void k_csr_scan(int *ptr, int V) {
    __shared__ int part[1024];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int chunk = (V + nth - 1) / nth;
    const int b = 1 + tid * chunk, e = min(V + 1, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += ptr[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int i = 0; i < nth; ++i) {
            const int q = part[i];
            part[i] = acc;
            acc += q;
        }
    }
    __syncthreads();
    int acc = part[tid];
    for (int i = b; i < e; ++i) {
        acc += ptr[i];
        ptr[i] = acc;
    }
}

__global__ void k_csr_fill(const int4 *__restrict__ tet, int T, int *cursor, int *idx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int4 a = tet[t];
    idx[atomicAdd(cursor + a.x, 1)] = 4 * t + 0;
    idx[atomicAdd(cursor + a.y, 1)] = 4 * t + 1;
    idx[atomicAdd(cursor + a.z, 1)] = 4 * t + 2;
    idx[atomicAdd(cursor + a.w, 1)] = 4 * t + 3;
}

// Rows were filled in arbitrary order; sort each ascending (rows are short).
__global__ void k_csr_sort(const int *__restrict__ ptr, int V, int *idx) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int b = ptr[v], e = ptr[v + 1];
    for (int i = b + 1; i < e; ++i) {
        const int key = idx[i];
        int j = i - 1;
        while (j >= b && idx[j] > key) {
            idx[j + 1] = idx[j];
            --j;
        }
        idx[j + 1] = key;
    }
}

cudaError_t launch_csr_build(const int4 *tet, int T, int V, int *ptr, int *idx, int *cursor, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ptr, 0, sizeof(int) * (size_t)(V + 1), s);
    if (e != cudaSuccess) return e;
    if (T > 0) k_csr_count<<<(T + 255) / 256, 256, 0, s>>>(tet, T, ptr);
    k_csr_scan<<<1, 1024, 0, s>>>(ptr, V);
    e = cudaMemcpyAsync(cursor, ptr, sizeof(int) * (size_t)V, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (T > 0) k_csr_fill<<<(T + 255) / 256, 256, 0, s>>>(tet, T, cursor, idx);
    if (V > 0) k_csr_sort<<<(V + 255) / 256, 256, 0, s>>>(ptr, V, idx);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host I/O
__global__ void k_set_positions(const double *__restrict__ y64, int v0, int nv, const double *__restrict__ xref64,
                                float4 *u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int g = v0 + i;
    u[g] = make_float4((float)(y64[3 * i] - xref64[3 * g]), (float)(y64[3 * i + 1] - xref64[3 * g + 1]),
                       (float)(y64[3 * i + 2] - xref64[3 * g + 2]), 0.f);
}

__global__ void k_get_positions(const float4 *__restrict__ u, const double *__restrict__ xref64, int v0, int nv,
                                double *y64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const int g = v0 + i;
    const float4 d = u[g];
    y64[3 * i] = xref64[3 * g] + (double)d.x;
    y64[3 * i + 1] = xref64[3 * g + 1] + (double)d.y;
    y64[3 * i + 2] = xref64[3 * g + 2] + (double)d.z;
}

__global__ void k_get_forces(const float4 *__restrict__ fv, int v0, int nv, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const float4 f = fv[v0 + i];
    out[3 * i] = f.x;
    out[3 * i + 1] = f.y;
    out[3 * i + 2] = f.z;
}

cudaError_t launch_set_positions(const double *y64, int v0, int nv, const double *xref64, float4 *u, cudaStream_t s) {
    if (nv > 0) k_set_positions<<<(nv + 255) / 256, 256, 0, s>>>(y64, v0, nv, xref64, u);
    return cudaGetLastError();
}

cudaError_t launch_get_positions(const float4 *u, const double *xref64, int v0, int nv, double *y64,
                                 cudaStream_t s) {
    if (nv > 0) k_get_positions<<<(nv + 255) / 256, 256, 0, s>>>(u, xref64, v0, nv, y64);
    return cudaGetLastError();
}

cudaError_t launch_get_forces(const float4 *fv, int v0, int nv, double *out, cudaStream_t s) {
    if (nv > 0) k_get_forces<<<(nv + 255) / 256, 256, 0, s>>>(fv, v0, nv, out);
    return cudaGetLastError();
}

__global__ void k_pack_tets(int T, const float *__restrict__ B, const float *__restrict__ V0,
                            const int *__restrict__ tmat, float4 *__restrict__ Bp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const float w[3] = {V0[t], __int_as_float(tmat[t]), 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k)
        Bp[k * T + t] = make_float4(B[(3 * k + 0) * T + t], B[(3 * k + 1) * T + t], B[(3 * k + 2) * T + t], w[k]);
}

cudaError_t launch_pack_tets(int T, const float *B, const float *V0, const int *tmat, float4 *Bp, cudaStream_t s) {
    if (T <= 0) return cudaSuccess;
    k_pack_tets<<<(T + 255) / 256, 256, 0, s>>>(T, B, V0, tmat, Bp);
    return cudaGetLastError();
}

__global__ void k_shift_slots(int T, int from, int delta, int *tmat) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T && tmat[t] >= from) tmat[t] += delta;
}

cudaError_t launch_shift_slots(int T, int from, int delta, int *tmat, cudaStream_t s) {
    if (T <= 0 || delta == 0) return cudaSuccess;
    k_shift_slots<<<(T + 255) / 256, 256, 0, s>>>(T, from, delta, tmat);
    return cudaGetLastError();
}

}  // namespace cf
