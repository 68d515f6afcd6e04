// Vertex forces without any device allocation (cf_vertex_forces_static).
//
// Some callers cannot allocate device memory: a solver embedded as a plugin
// in a host application that owns every device buffer, or a real-time loop
// whose memory is fixed up front. This entry point takes the caller's device
// buffers for inputs and outputs and keeps its one piece of scratch - the
// per-corner forces between the tet kernel and the vertex sums - in a
// fixed-size array of static device memory, reserved on every GPU that loads
// the library until the process exits.
//
// Host code cannot use the name of a __device__ array as a device address,
// so the set-up looks the addresses up with cudaGetSymbolAddress, with the
// device current, and caches them per device. The cache is keyed on the
// unique id of the device's current CUDA context (cuCtxGetId, reached
// through the runtime's driver entry points): if the context is destroyed
// (cudaDeviceReset) and created again, the module is loaded anew, its arrays
// may move, and the next call looks them up again. Without that driver
// entry point every call looks them up.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cellfsi.h"
#include "internal.cuh"

using namespace cf;

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) float4 g_corner[4 * CF_STATIC_MAX_TETS];  // corner forces [4][nt]
static __device__ __align__(256) int g_tcell[CF_STATIC_MAX_TETS];           // never written: all zero
static __device__ __align__(256) float4 g_mat[1];                          // mu1, mu2, kappa, 0
static __device__ __align__(256) unsigned g_err[1];                        // device error word

struct StaticAddr {
    bool ready = false;
    unsigned long long ctx_id = 0;  // context the addresses belong to
    float4 *corner = nullptr;
    int *tcell = nullptr;
    float4 *mat = nullptr;
    unsigned *err = nullptr;
};

StaticAddr g_addr[kMaxDevices];
std::mutex g_lock;

using CtxGetCurrent = CUresult (*)(CUcontext *);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrent g_get_current = nullptr;
CtxGetId g_get_id = nullptr;
std::once_flag g_entry_once;

// Unique id of the calling thread's current context; false if the driver
// entry points are unavailable or no context is current.
bool current_context_id(unsigned long long *id) {
    std::call_once(g_entry_once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            g_get_current = reinterpret_cast<CtxGetCurrent>(a);
            g_get_id = reinterpret_cast<CtxGetId>(b);
        }
        cudaGetLastError();  // a failed lookup leaves no sticky state behind
    });
    if (!g_get_current || !g_get_id) return false;
    CUcontext ctx = nullptr;
    if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_get_id(ctx, id) == CUDA_SUCCESS;
}

// Set-up once per device and context, with that device current.
cf_status static_setup(int dev, StaticAddr &out) {
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);  // false before the runtime made a context current
    std::lock_guard<std::mutex> lk(g_lock);
    StaticAddr &a = g_addr[dev];
    if (!a.ready || !have_id || a.ctx_id != id) {
        a.ready = false;
        if (cudaGetSymbolAddress((void **)&a.corner, g_corner) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&a.tcell, g_tcell) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&a.mat, g_mat) != cudaSuccess ||
            cudaGetSymbolAddress((void **)&a.err, g_err) != cudaSuccess)
            return CF_ECUDA;
        // the lookups made the device's context current if none was: the
        // addresses belong to that context
        have_id = current_context_id(&id);
        a.ctx_id = id;
        a.ready = have_id;  // without an id, look up again next call
    }
    out = a;
    return CF_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" cf_status cf_vertex_forces_static(int32_t nv, int32_t nt, const int32_t *tets, const float *B,
                                             const float *V0, const float *u, const int32_t *csr_ptr,
                                             const int32_t *csr_idx, double mu, double kappa, double w, float *f,
                                             void *cuda_stream) {
    if (nv < 1 || nt < 1 || nt > CF_STATIC_MAX_TETS) return CF_EINVAL;
    if (!tets || !B || !V0 || !u || !csr_ptr || !csr_idx || !f) return CF_EINVAL;
    if (!aligned16(tets) || !aligned16(u) || !aligned16(f)) return CF_EINVAL;
    if (!(mu >= 0.0 && kappa >= 0.0 && w >= 0.0 && w <= 1.0)) return CF_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CF_ECUDA;
    StaticAddr a;
    if (static_setup(dev, a) != CF_OK) return CF_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    const float4 mat = make_float4((float)(w * mu), (float)((1.0 - w) * mu), (float)kappa, 0.f);
    if (cudaMemcpyAsync(a.mat, &mat, sizeof mat, cudaMemcpyHostToDevice, s) != cudaSuccess) return CF_ECUDA;
    if (cudaMemsetAsync(a.err, 0, sizeof(unsigned), s) != cudaSuccess) return CF_ECUDA;

    MeshView m{};
    m.V = nv;
    m.T = nt;
    m.tet = reinterpret_cast<const int4 *>(tets);
    m.B = B;
    m.V0 = V0;
    m.tcell = a.tcell;
    m.mat = a.mat;
    m.csr_ptr = csr_ptr;
    m.csr_idx = csr_idx;
    m.fc = a.corner;
    m.fv = reinterpret_cast<float4 *>(f);
    const float4 *u4 = reinterpret_cast<const float4 *>(u);
    if (launch_tet_force(m, u4, a.err, s) != cudaSuccess) return CF_ECUDA;
    if (launch_gather_spread(m, u4, nullptr, nullptr, a.err, s) != cudaSuccess) return CF_ECUDA;

    unsigned h = 0;
    if (cudaMemcpyAsync(&h, a.err, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CF_ECUDA;
    if (h & ERR_INVERTED) return CF_EINVERTED;
    if (h & ERR_NONFINITE) return CF_ENONFINITE;
    return CF_OK;
}
