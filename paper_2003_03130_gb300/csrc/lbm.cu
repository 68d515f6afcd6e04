// K4: D3Q19 lattice-Boltzmann stream + collide (the fluid of Sec. 6; the
// paper uses ESPResSo's LB without stating the operator). Pull scheme: the
// buffer holds post-collision populations, a node pulls f_q(x - c_q) from the
// old buffer, collides, and writes the new post-collision populations at x
// into the other buffer.
//
//   walls (Sec. 6.1 moving planes): a pull from beyond y = -1/2 or
//     y = ny - 1/2 is halfway bounce-back with the moving-wall term,
//     f_q(x) = f*_opp(q)(x) + 6 w_q (c_q . u_wall)  (rho_0 = 1);
//   moments: rho = 1 + sum d_q, rho u = sum c_q d_q + F/2, F = F(x) + g;
//   BGK + Guo: d*_q = d_q + omega (d^eq_q - d_q)
//                     + (1 - omega/2) w_q [3 (c_q - u) + 9 (c_q . u) c_q] . F,
//     d^eq_q = w_q [(rho - 1) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u)].
//
// Storage: populations are kept as deviations d_q = f_q - w_q from the rest
// equilibrium (FP32 rounding then scales with the O(u) signal), in FP32, or in
// FP16 / BF16 multiplied by a power of two per weight class (2^14, 2^16, 2^17
// for w = 1/3, 1/18, 1/36, so that the stored values are O(10^3) and never
// subnormal in FP16); the collide always runs in FP32. Population loads and
// stores carry the streaming cache hint (evict first): every population is
// touched once per step, and the hint keeps the cells' few MB of mesh data
// resident in L2 while the lattice streams through it.
//
// One node per thread: 19 independent coalesced loads per node (x-shifted
// rows are off by one word; neighbouring warps share the lines in L2), the
// collide, 19 coalesced stores. The 16-bit formats also come in a pair form
// (two x-neighbours per thread, 32-bit population access, packed FP32
// collide; see "node pairs" below). The whole-lattice and far-field kernels take
// rows of 128 nodes along x; with cells the lattice is also cut into tiles of
// 256 nodes (x fastest), the unit of the force region, and the near field
// runs half a tile of the region per block and work item.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.cuh"

namespace cf {

// ---------------------------------------------------------------- storage
// ld / st: streaming loads and stores with round-to-nearest conversion;
// st_sr: stochastic rounding to the 16-bit format, the dither being random
// bits below the last kept mantissa bit (13 bits for FP16, 16 for BF16).
// Adding them to the FP32 pattern and truncating rounds the magnitude up
// with probability equal to the dropped fraction, so the rounding is
// unbiased (exact for FP16-normal values). The caller passes a zero dither
// for non-finite values, which then convert as they are.
template <class T>
struct Pop;

// FP32 also comes in an L2-normal form (CS false: loads and stores cached in
// L2 with normal priority, not in L1), which keeps more of a large lattice's
// populations in L2 between the far and near fields; the streaming form
// protects the cell data instead. The launch shape picks one.
template <>
struct Pop<float> {
    static constexpr int kDropped = 0;
    template <bool CS = true>
    static __device__ __forceinline__ float ld(const float *p) {
        return CS ? __ldcs(p) : __ldcg(p);
    }
    template <bool CS = true>
    static __device__ __forceinline__ void st(float *p, float v) {
        if (CS)
            __stcs(p, v);
        else
            __stcg(p, v);
    }
    template <bool CS = true>
    static __device__ __forceinline__ void st_sr(float *p, float v, unsigned) {
        st<CS>(p, v);
    }
};

template <>
struct Pop<__half> {
    static constexpr int kDropped = 13;
    template <bool CS = true>
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldcs(p)); }
    template <bool CS = true>
    static __device__ __forceinline__ void st(__half *p, float v) { __stcs(p, __float2half_rn(v)); }
    template <bool CS = true>
    static __device__ __forceinline__ void st_sr(__half *p, float v, unsigned dither) {
        __stcs(p, __float2half_rz(__uint_as_float(__float_as_uint(v) + dither)));
    }
};

template <>
struct Pop<__nv_bfloat16> {
    static constexpr int kDropped = 16;
    template <bool CS = true>
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldcs(p)); }
    template <bool CS = true>
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { __stcs(p, __float2bfloat16_rn(v)); }
    template <bool CS = true>
    static __device__ __forceinline__ void st_sr(__nv_bfloat16 *p, float v, unsigned dither) {
        __stcs(p, __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + dither)));
    }
};

// Random bits for the dither: h = mix32(n ^ mix32(seed)) per node with the
// "lowbias32" xorshift-multiply finaliser (C. Wellons, "Prospecting for hash
// functions", 2018); population q takes the top bits of the Weyl step
// h + q * 0x9e3779b9 (uniform for every q, independent across steps through
// the seed).
__device__ __forceinline__ unsigned mix32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// stored value = d_q * scale; exact powers of two
template <class T>
__device__ __forceinline__ constexpr float pop_scale(int q) {
    return sizeof(T) == 4 ? 1.f : (q == 0 ? 16384.f : (q <= 6 ? 65536.f : 131072.f));
}
template <class T>
__device__ __forceinline__ constexpr float pop_unscale(int q) {
    return sizeof(T) == 4 ? 1.f : (q == 0 ? 1.f / 16384.f : (q <= 6 ? 1.f / 65536.f : 1.f / 131072.f));
}

// ---------------------------------------------------------------- collide
// c . v for a compile-time lattice vector (a, b, c): only the nonzero
// components enter (0.0f * v cannot be folded away under IEEE rules).
template <int a, int b, int c>
__device__ __forceinline__ float cdot(float x, float y, float z) {
    float s = 0.f;
    if constexpr (a != 0 && b != 0) {
        s = (a > 0 ? x : -x) + (b > 0 ? y : -y);
    } else if constexpr (a != 0 && c != 0) {
        s = (a > 0 ? x : -x) + (c > 0 ? z : -z);
    } else if constexpr (b != 0 && c != 0) {
        s = (b > 0 ? y : -y) + (c > 0 ? z : -z);
    } else if constexpr (a != 0) {
        s = a > 0 ? x : -x;
    } else if constexpr (b != 0) {
        s = b > 0 ? y : -y;
    } else if constexpr (c != 0) {
        s = c > 0 ? z : -z;
    }
    return s;
}

// Per weight class w: constants of the collision that do not depend on the
// direction within the class.
struct WClass {
    float c0;   // omega (w drho - w rho 3/2 u.u) - 3 g w (u.F): direction-free part
    float e45;  // 9/2 omega w rho
    float o3;   // 3 omega w rho
    float g9;   // 9 g w
    float g3;   // 3 g w
};

__device__ __forceinline__ WClass wclass(float w, float drho, float rho, float usq15, float uF, float om, float g) {
    WClass k;
    const float wr = w * rho;
    k.c0 = om * (w * drho - wr * usq15) - 3.f * g * w * uF;
    k.e45 = 4.5f * om * wr;
    k.o3 = 3.f * om * wr;
    k.g9 = 9.f * g * w;
    k.g3 = 3.f * g * w;
    return k;
}

// Collide the opposite pair (A, opp(A)) in place. With cu = c_A.u and
// cF = c_A.F the equilibrium and source split into a part even in c (P) and a
// part odd in c (Q): d*_A = (1-omega) d_A + P + Q, d*_opp = (1-omega) d_opp +
// P - Q, with
//   P = omega w [drho + rho (9/2 cu^2 - 3/2 u.u)] + g w [9 cu cF - 3 u.F],
//   Q = 3 omega w rho cu + 3 g w cF.
template <int A>
__device__ __forceinline__ void collide_pair(float (&d)[19], const WClass &k, float om1, float ux, float uy, float uz,
                                             float Fx, float Fy, float Fz) {
    constexpr int B = opp(A);
    const float cu = cdot<cx(A), cy(A), cz(A)>(ux, uy, uz);
    const float cF = cdot<cx(A), cy(A), cz(A)>(Fx, Fy, Fz);
    const float P = fmaf(cu, fmaf(k.g9, cF, k.e45 * cu), k.c0);
    const float Q = fmaf(k.o3, cu, k.g3 * cF);
    const float a = fmaf(om1, d[A], P + Q);
    const float b = fmaf(om1, d[B], P - Q);
    d[A] = a;
    d[B] = b;
}

// Moments and collision of one node, in place, in stored units: d holds the
// pulled populations as stored (d_q times its class scale S) on entry and the
// post-collision ones, scaled the same way, on exit. The moments sum each
// weight class first and unscale the three sums; the collision constants are
// those of the weights w S. S is a power of two, so both are exact
// rescalings of the same operations on the unscaled values, and no
// population is multiplied by its scale on load or store. Returns u(t).
template <class T>
__device__ __forceinline__ float3 collide(float (&d)[19], float Fx, float Fy, float Fz, const LbmParams &p) {
    constexpr float s0 = pop_scale<T>(0), s1 = pop_scale<T>(1), s2 = pop_scale<T>(7);
    const float face = ((d[1] + d[2]) + (d[3] + d[4])) + (d[5] + d[6]);
    const float edge = ((d[7] + d[8]) + (d[9] + d[10])) + ((d[11] + d[12]) + (d[13] + d[14])) +
                       ((d[15] + d[16]) + (d[17] + d[18]));
    const float drho = fmaf(edge, 1.f / s2, fmaf(face, 1.f / s1, d[0] * (1.f / s0)));
    // x: +1 at 1, 15..18; -1 at 2, 7..10
    const float ex = ((d[15] - d[7]) + (d[16] - d[8])) + ((d[17] - d[9]) + (d[18] - d[10]));
    // y: +1 at 3, 10, 13, 14, 18; -1 at 4, 7, 11, 12, 15
    const float ey = ((d[10] - d[7]) + (d[13] - d[11])) + ((d[14] - d[12]) + (d[18] - d[15]));
    // z: +1 at 5, 9, 12, 14, 17; -1 at 6, 8, 11, 13, 16
    const float ez = ((d[9] - d[8]) + (d[12] - d[11])) + ((d[14] - d[13]) + (d[17] - d[16]));
    const float jx = fmaf(ex, 1.f / s2, (d[1] - d[2]) * (1.f / s1));
    const float jy = fmaf(ey, 1.f / s2, (d[3] - d[4]) * (1.f / s1));
    const float jz = fmaf(ez, 1.f / s2, (d[5] - d[6]) * (1.f / s1));
    const float rho = 1.f + drho;
    const float ir = __frcp_rn(rho);
    const float ux = fmaf(0.5f, Fx, jx) * ir, uy = fmaf(0.5f, Fy, jy) * ir, uz = fmaf(0.5f, Fz, jz) * ir;
    const float usq15 = 1.5f * fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float uF = fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz));
    const float om = p.omega, g = p.guo, om1 = 1.f - om;
    const WClass k0 = wclass((1.f / 3.f) * s0, drho, rho, usq15, uF, om, g);
    const WClass k1 = wclass((1.f / 18.f) * s1, drho, rho, usq15, uF, om, g);
    const WClass k2 = wclass((1.f / 36.f) * s2, drho, rho, usq15, uF, om, g);
    d[0] = fmaf(om1, d[0], k0.c0);
    collide_pair<1>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<3>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<5>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<7>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<8>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<9>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<10>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<11>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair<12>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    return make_float3(ux, uy, uz);
}

// pull from beyond a wall? (only in rows y = 0 and y = ny - 1)
template <int q>
__device__ __forceinline__ bool wall_pull(int y, int ny) {
    return (cy(q) == 1 && y == 0) || (cy(q) == -1 && y == ny - 1);
}

// ---------------------------------------------------------------- one node
// store = false: load and collide but write nothing (a node found, after its
// loads were issued, to belong to the other part of the split).
template <class T, bool WALL, bool HAS_F, bool CS = true>
__device__ __forceinline__ void lbm_node(const T *__restrict__ fin, T *__restrict__ fout,
                                         float4 *__restrict__ F, const LbmParams &p, int x, int y, int z,
                                         float4 *__restrict__ vel, unsigned seed, bool store = true) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;  // 64-bit population offsets q * N + n
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int n = x + nx * (y + ny * z);

    float d[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : x);
        const int sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z);
        const int sy = y - cy(q);
        if (WALL && ((cy(q) == 1 && y == 0) || (cy(q) == -1 && y == ny - 1))) {
            const float uw = cy(q) == 1 ? p.uw_lo : p.uw_hi;
            d[q] = Pop<T>::template ld<CS>(fin + opp(q) * N + n);
            if (cx(q) != 0) d[q] += (6.f * wq(q) * cx(q) * pop_scale<T>(q)) * uw;
        } else {
            d[q] = Pop<T>::template ld<CS>(fin + q * N + sx + nx * (sy + ny * sz));
        }
    }
    float Fx = p.gx, Fy = p.gy, Fz = p.gz;
    bool spread = false;
    if (HAS_F) {
        const float4 a = force_at(F, p, n, spread);
        Fx += a.x;
        Fy += a.y;
        Fz += a.z;
    }
    const float3 u = collide<T>(d, Fx, Fy, Fz, p);
    if (!store) return;
    if (HAS_F && spread) force_clear(F, p, n);  // consumed: the next step spreads onto zeros
    if (vel) {  // u(t) of this step, for the interpolation at the vertices
        vel[n] = make_float4(u.x, u.y, u.z, 0.f);
    }
    if constexpr (sizeof(T) == 2) {
        if (p.sr) {
            const unsigned h = mix32((unsigned)n ^ mix32(seed));
            // a non-finite node (any NaN input makes u NaN) converts without dither
            const unsigned mask = isfinite(u.x + u.y + u.z) ? (1u << Pop<T>::kDropped) - 1u : 0u;
#pragma unroll
            for (int q = 0; q < 19; ++q) {
                const unsigned r = (h + (unsigned)q * 0x9e3779b9u) >> (32 - Pop<T>::kDropped);
                Pop<T>::template st_sr<CS>(fout + q * N + n, d[q], r & mask);
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 19; ++q) Pop<T>::template st<CS>(fout + q * N + n, d[q]);
}

// ---------------------------------------------------------------- node pairs
// 16-bit storage, two neighbouring nodes (x0, x0 + 1) per thread, x0 even
// (nx even): one 32-bit load or store moves a population of both nodes, and
// the collide runs on packed FP32 pairs (f32x2 arithmetic, sm_100 and
// later), so that a thread issues about half the instructions per node of
// the one-node form (which is bound by instruction issue at 2 bytes per
// population, not by HBM). A pull along x (c_x = +1: from x - 1; c_x = -1:
// from x + 1) straddles two aligned pairs of the source row: both are loaded
// (the second lies in the same L1/L2 sectors as a neighbouring thread's) and
// the middle two values are taken with one byte permute. Both nodes of a
// pair lie in the same force-region tile (tiles are at least 8 nodes wide
// in x).
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&d);
}

// c . v for a lattice vector whose first nonzero component is +1 (only
// nonzero components enter).
template <int a, int b, int c>
__device__ __forceinline__ float2 cdot2(float2 x, float2 y, float2 z) {
    static_assert(a > 0 || (a == 0 && b > 0) || (a == 0 && b == 0 && c > 0), "first component must be +1");
    if constexpr (a != 0 && b != 0) return b > 0 ? add2(x, y) : sub2(x, y);
    else if constexpr (a != 0 && c != 0) return c > 0 ? add2(x, z) : sub2(x, z);
    else if constexpr (b != 0 && c != 0) return c > 0 ? add2(y, z) : sub2(y, z);
    else if constexpr (a != 0) return x;
    else if constexpr (b != 0) return y;
    else return z;
}

__host__ __device__ constexpr int first_nonzero(int q) { return cx(q) != 0 ? cx(q) : cy(q) != 0 ? cy(q) : cz(q); }

struct WClass2 {
    float2 c0, e45, o3;
    float g9, g3;
};

__device__ __forceinline__ WClass2 wclass2(float w, float2 drho, float2 rho, float2 usq15, float2 uF, float om, float g) {
    WClass2 k;
    const float2 wr = mul2(f2(w), rho);
    k.c0 = fma2(f2(-3.f * g * w), uF, mul2(f2(om), sub2(mul2(f2(w), drho), mul2(wr, usq15))));
    k.e45 = mul2(f2(4.5f * om), wr);
    k.o3 = mul2(f2(3.f * om), wr);
    k.g9 = 9.f * g * w;
    k.g3 = 3.f * g * w;
    return k;
}

// The pair (A, opp(A)) of both nodes, as collide_pair, with the sign of c
// chosen so that its first nonzero component is +1 (P is even in c, Q odd).
template <int A>
__device__ __forceinline__ void collide_pair2(float2 (&d)[19], const WClass2 &k, float2 om1, float2 ux, float2 uy,
                                              float2 uz, float2 Fx, float2 Fy, float2 Fz) {
    constexpr int Ap = first_nonzero(A) > 0 ? A : opp(A), Bp = opp(Ap);
    const float2 cu = cdot2<cx(Ap), cy(Ap), cz(Ap)>(ux, uy, uz);
    const float2 cF = cdot2<cx(Ap), cy(Ap), cz(Ap)>(Fx, Fy, Fz);
    const float2 P = fma2(cu, fma2(f2(k.g9), cF, mul2(k.e45, cu)), k.c0);
    const float2 Q = fma2(k.o3, cu, mul2(f2(k.g3), cF));
    const float2 a = fma2(om1, d[Ap], add2(P, Q));
    const float2 b = fma2(om1, d[Bp], sub2(P, Q));
    d[Ap] = a;
    d[Bp] = b;
}

// collide<T> for two nodes at once (the same operations per node, in packed
// arithmetic); returns u(t) of both.
template <class T>
__device__ __forceinline__ void collide2(float2 (&d)[19], float2 Fx, float2 Fy, float2 Fz, const LbmParams &p,
                                         float2 &ux, float2 &uy, float2 &uz) {
    constexpr float s0 = pop_scale<T>(0), s1 = pop_scale<T>(1), s2 = pop_scale<T>(7);
    const float2 face = add2(add2(add2(d[1], d[2]), add2(d[3], d[4])), add2(d[5], d[6]));
    const float2 edge = add2(add2(add2(add2(d[7], d[8]), add2(d[9], d[10])), add2(add2(d[11], d[12]), add2(d[13], d[14]))),
                             add2(add2(d[15], d[16]), add2(d[17], d[18])));
    const float2 drho = fma2(edge, f2(1.f / s2), fma2(face, f2(1.f / s1), mul2(d[0], f2(1.f / s0))));
    const float2 ex = add2(add2(sub2(d[15], d[7]), sub2(d[16], d[8])), add2(sub2(d[17], d[9]), sub2(d[18], d[10])));
    const float2 ey = add2(add2(sub2(d[10], d[7]), sub2(d[13], d[11])), add2(sub2(d[14], d[12]), sub2(d[18], d[15])));
    const float2 ez = add2(add2(sub2(d[9], d[8]), sub2(d[12], d[11])), add2(sub2(d[14], d[13]), sub2(d[17], d[16])));
    const float2 jx = fma2(ex, f2(1.f / s2), mul2(sub2(d[1], d[2]), f2(1.f / s1)));
    const float2 jy = fma2(ey, f2(1.f / s2), mul2(sub2(d[3], d[4]), f2(1.f / s1)));
    const float2 jz = fma2(ez, f2(1.f / s2), mul2(sub2(d[5], d[6]), f2(1.f / s1)));
    const float2 rho = add2(f2(1.f), drho);
    const float2 ir = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
    ux = mul2(fma2(f2(0.5f), Fx, jx), ir);
    uy = mul2(fma2(f2(0.5f), Fy, jy), ir);
    uz = mul2(fma2(f2(0.5f), Fz, jz), ir);
    const float2 usq15 = mul2(f2(1.5f), fma2(ux, ux, fma2(uy, uy, mul2(uz, uz))));
    const float2 uF = fma2(ux, Fx, fma2(uy, Fy, mul2(uz, Fz)));
    const float om = p.omega, g = p.guo;
    const float2 om1 = f2(1.f - om);
    const WClass2 k0 = wclass2((1.f / 3.f) * s0, drho, rho, usq15, uF, om, g);
    const WClass2 k1 = wclass2((1.f / 18.f) * s1, drho, rho, usq15, uF, om, g);
    const WClass2 k2 = wclass2((1.f / 36.f) * s2, drho, rho, usq15, uF, om, g);
    d[0] = fma2(om1, d[0], k0.c0);
    collide_pair2<1>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<3>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<5>(d, k1, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<7>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<8>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<9>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<10>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<11>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
    collide_pair2<12>(d, k2, om1, ux, uy, uz, Fx, Fy, Fz);
}

// 32-bit pair access: the raw bits of two 16-bit populations (lower half =
// the even node), their FP32 values, and the rounded or stochastically
// rounded conversion back.
__device__ __forceinline__ unsigned ld_pair(const void *p) { return __ldcs(static_cast<const unsigned *>(p)); }
__device__ __forceinline__ void st_pair(void *p, unsigned v) { __stcs(static_cast<unsigned *>(p), v); }

template <class T>
__device__ __forceinline__ float2 unpack2(unsigned w);
template <>
__device__ __forceinline__ float2 unpack2<__half>(unsigned w) {
    return make_float2(__half2float(__ushort_as_half((unsigned short)(w & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(w >> 16))));
}
template <>
__device__ __forceinline__ float2 unpack2<__nv_bfloat16>(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Round to nearest: one packing conversion for both values.
template <class T>
__device__ __forceinline__ unsigned pack2_rn(float2 v);
template <>
__device__ __forceinline__ unsigned pack2_rn<__half>(float2 v) {
    unsigned d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.y), "f"(v.x));
    return d;
}
template <>
__device__ __forceinline__ unsigned pack2_rn<__nv_bfloat16>(float2 v) {
    unsigned d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.y), "f"(v.x));
    return d;
}

// Stochastic rounding of both values by the hardware conversion (cvt.rs,
// sm_100a and later): each value rounds away from zero with probability
// equal to the dropped fraction of its last kept unit, the odd node's value
// drawing on the upper 16 bits of r, the even node's on the lower 16 (of
// which FP16 uses 13). Measured on GB300: a value 0.7 (0.3) of a unit above
// a representable one rounds up with frequency 0.7002 (0.3002) over 2^20
// random words, in both formats.
template <class T>
__device__ __forceinline__ unsigned pack2_sr(float2 v, unsigned r) {
    unsigned d;
    if constexpr (std::is_same<T, __half>::value)
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(r));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(r));
    return d;
}

// Nodes (x0, x0 + 1) of row (y, z): pull, collide, store, as lbm_node.
template <class T, bool WALL, bool HAS_F>
__device__ __forceinline__ void lbm_pair(const T *__restrict__ fin, T *__restrict__ fout, float4 *__restrict__ F,
                                         const LbmParams &p, int x0, int y, int z, float4 *__restrict__ vel,
                                         unsigned seed) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;  // 64-bit population offsets q * N + n
    const int xm = x0 == 0 ? nx - 2 : x0 - 2, xp = x0 + 2 == nx ? 0 : x0 + 2;  // neighbouring pairs
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int n0 = x0 + nx * (y + ny * z);

    float2 d[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z);
        const int sy = y - cy(q);
        if (WALL && ((cy(q) == 1 && y == 0) || (cy(q) == -1 && y == ny - 1))) {
            const float uw = cy(q) == 1 ? p.uw_lo : p.uw_hi;
            d[q] = unpack2<T>(ld_pair(fin + opp(q) * N + n0));
            if (cx(q) != 0) d[q] = add2(d[q], f2((6.f * wq(q) * cx(q) * pop_scale<T>(q)) * uw));
        } else {
            const T *row = fin + q * N + nx * (sy + ny * sz);
            unsigned w;
            if (cx(q) == 1)
                w = __byte_perm(ld_pair(row + xm), ld_pair(row + x0), 0x5432);  // (x0 - 1, x0)
            else if (cx(q) == -1)
                w = __byte_perm(ld_pair(row + x0), ld_pair(row + xp), 0x5432);  // (x0 + 1, x0 + 2)
            else
                w = ld_pair(row + x0);
            d[q] = unpack2<T>(w);
        }
    }
    float2 Fx = f2(p.gx), Fy = f2(p.gy), Fz = f2(p.gz);
    bool spread0 = false, spread1 = false;
    if (HAS_F) {
        const float4 a = force_at(F, p, n0, spread0), b = force_at(F, p, n0 + 1, spread1);
        Fx = add2(Fx, make_float2(a.x, b.x));
        Fy = add2(Fy, make_float2(a.y, b.y));
        Fz = add2(Fz, make_float2(a.z, b.z));
    }
    float2 ux, uy, uz;
    collide2<T>(d, Fx, Fy, Fz, p, ux, uy, uz);
    if (HAS_F) {  // consumed: the next step spreads onto zeros
        if (spread0) force_clear(F, p, n0);
        if (spread1) force_clear(F, p, n0 + 1);
    }
    if (vel) {
        vel[n0] = make_float4(ux.x, uy.x, uz.x, 0.f);
        vel[n0 + 1] = make_float4(ux.y, uy.y, uz.y, 0.f);
    }
    if (p.sr) {
        // random bits per pair and population: the Weyl step h + q 0x9e3779b9
        // of a per-pair hash of the node and the step's seed
        const unsigned h = mix32((unsigned)n0 ^ mix32(seed));
#pragma unroll
        for (int q = 0; q < 19; ++q) st_pair(fout + q * N + n0, pack2_sr<T>(d[q], h + (unsigned)q * 0x9e3779b9u));
        return;
    }
#pragma unroll
    for (int q = 0; q < 19; ++q) st_pair(fout + q * N + n0, pack2_rn<T>(d[q]));
}

// ---------------------------------------------------------------- kernels
// Whole lattice, no force field (fluid-only runs).
template <class T>
__global__ void __launch_bounds__(128) k_lbm(const T *__restrict__ fin, T *__restrict__ fout, LbmParams p,
                                             const unsigned *__restrict__ seed_in, unsigned *__restrict__ seed_out) {
    const unsigned seed = *seed_in;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *seed_out = seed + 1u;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    if (y > 0 && y < p.ny - 1)
        lbm_node<T, false, false>(fin, fout, nullptr, p, x, y, z, nullptr, seed);
    else
        lbm_node<T, true, false>(fin, fout, nullptr, p, x, y, z, nullptr, seed);
}

// Node of thread i in tile (tx, ty, tz): x fastest within the tile. False if
// the node lies outside the lattice (partial tiles at the upper ends).
__device__ __forceinline__ bool tile_node(const LbmParams &p, int tx, int ty, int tz, int i, int &x, int &y, int &z) {
    x = (tx << p.tlx) + (i & ((1 << p.tlx) - 1));
    y = (ty << p.tly) + ((i >> p.tlx) & ((1 << p.tly) - 1));
    z = (tz << p.tlz) + (i >> (p.tlx + p.tly));
    return x < p.nx && y < p.ny && z < p.nz;
}

// Near field: half a tile per block, 128 threads, one node each.
constexpr int kTileBlock = kTileNodes / 2;

// The nodes outside the force region (F is zero there: no force-field
// read), in rows of 128 nodes along x as in the fluid-only kernel, so that y
// and z stay uniform over a block; a thread whose node lies in a region tile
// returns at once.
// SPEC: the region test resolves while the populations load (a region
// node's loads are wasted, a far node saves a round trip before its loads);
// otherwise a region node returns before loading.
template <class T, bool SPEC, bool CS = true>
__global__ void __launch_bounds__(128) k_lbm_far(const T *__restrict__ fin, T *__restrict__ fout, LbmParams p,
                                                 const unsigned *__restrict__ bits,
                                                 const unsigned *__restrict__ seed_in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const bool region = region_has(bits, tile_index(p, x >> p.tlx, y >> p.tly, z >> p.tlz));
    if (!SPEC && region) return;
    const unsigned seed = *seed_in;
    if (y > 0 && y < p.ny - 1)
        lbm_node<T, false, false, CS>(fin, fout, nullptr, p, x, y, z, nullptr, seed, !region);
    else
        lbm_node<T, true, false, CS>(fin, fout, nullptr, p, x, y, z, nullptr, seed, !region);
}

// The force region's nodes in rows of 128 along x over the whole lattice (the
// far field's layout: y and z uniform over a block); threads outside the
// region return at once. Cheaper per node than the list form when the region
// is a large part of the lattice.
template <class T, bool CS = true>
__global__ void __launch_bounds__(128) k_lbm_near_rows(const T *__restrict__ fin, T *__restrict__ fout,
                                                       float4 *__restrict__ F, LbmParams p,
                                                       const unsigned *__restrict__ bits, float4 *__restrict__ vel,
                                                       const unsigned *__restrict__ seed_in,
                                                       unsigned *__restrict__ seed_out) {
    const unsigned seed = *seed_in;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *seed_out = seed + 1u;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    if (!region_has(bits, tile_index(p, x >> p.tlx, y >> p.tly, z >> p.tlz))) return;
    if (y > 0 && y < p.ny - 1)
        lbm_node<T, false, true, CS>(fin, fout, F, p, x, y, z, vel, seed);
    else
        lbm_node<T, true, true, CS>(fin, fout, F, p, x, y, z, vel, seed);
}

// The force region's tiles, with the force field; also stores u(t) there.
// The grid is fixed when a step is captured while the region moves with the
// cells, so blocks stride over the region's half tiles. The tiles are the
// set bits of the region bitset: every block first forms, in shared memory,
// the running count of set bits before each bitset word (nwords + 1
// entries); the k-th tile of the region is then found by a binary search
// over those counts and a scan of one word.
template <class T, bool CS = true>
__global__ void __launch_bounds__(kTileBlock, 8) k_lbm_near(const T *__restrict__ fin, T *__restrict__ fout,
                                                            float4 *__restrict__ F, LbmParams p,
                                                            const unsigned *__restrict__ bits, int nwords,
                                                            float4 *__restrict__ vel,
                                                            const unsigned *__restrict__ seed_in,
                                                            unsigned *__restrict__ seed_out) {
    extern __shared__ int before[];  // [nwords + 1]: set bits in the words before word j
    __shared__ int warp_sum[kTileBlock / 32];
    const unsigned seed = *seed_in;
    if ((blockIdx.x | threadIdx.x) == 0) *seed_out = seed + 1u;
    // running counts: thread i takes a contiguous chunk of words
    const int chunk = (nwords + kTileBlock - 1) / kTileBlock, w0 = threadIdx.x * chunk;
    int mine = 0;
    for (int j = w0; j < w0 + chunk && j < nwords; ++j) mine += __popc(bits[j]);
    int incl = mine;  // inclusive scan over the block
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    int base = 0;
    for (int k = 0; k < wid; ++k) base += warp_sum[k];
    int run = base + incl - mine;
    for (int j = w0; j < w0 + chunk && j < nwords; ++j) {
        before[j] = run;
        run += __popc(bits[j]);
    }
    if (threadIdx.x == kTileBlock - 1) before[nwords] = run;
    __syncthreads();
    const int halves = 2 * before[nwords];
    for (int w = blockIdx.x; w < halves; w += gridDim.x) {
        const int rank = w >> 1;
        int lo = 0, hi = nwords - 1;  // the last word j with before[j] <= rank
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (before[mid] <= rank) lo = mid;
            else hi = mid - 1;
        }
        unsigned word = bits[lo];
        for (int k = rank - before[lo]; k > 0; --k) word &= word - 1u;  // drop the lower set bits
        const int tile = 32 * lo + __ffs(word) - 1;
        const int tx = tile % p.ntx, r = tile / p.ntx;
        int x, y, z;
        if (!tile_node(p, tx, r % p.nty, r / p.nty, (w & 1) * kTileBlock + threadIdx.x, x, y, z)) continue;
        if (y > 0 && y < p.ny - 1)
            lbm_node<T, false, true, CS>(fin, fout, F, p, x, y, z, vel, seed);
        else
            lbm_node<T, true, true, CS>(fin, fout, F, p, x, y, z, vel, seed);
    }
}

// ---------------------------------------------------------------- pair kernels
// The 16-bit storage formats with nx even: the whole-lattice, far-field and
// row-form near-field kernels with two nodes per thread (lbm_pair), rows of
// up to 64 pairs per block so that y and z stay uniform over a block. The
// whole-lattice and far-field forms are held to 72 registers (14 blocks per
// SM, a 16-byte spill): FP16-SR far field at 128^3 32.9 us against 34.3 us
// at 80 registers and 34.5 us at 64 (an 84-byte spill).
template <class T>
__global__ void __launch_bounds__(64, 14) k_lbm_pairs(const T *__restrict__ fin, T *__restrict__ fout, LbmParams p,
                                                  const unsigned *__restrict__ seed_in,
                                                  unsigned *__restrict__ seed_out) {
    const unsigned seed = *seed_in;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *seed_out = seed + 1u;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    if (y > 0 && y < p.ny - 1)
        lbm_pair<T, false, false>(fin, fout, nullptr, p, x0, y, z, nullptr, seed);
    else
        lbm_pair<T, true, false>(fin, fout, nullptr, p, x0, y, z, nullptr, seed);
}

template <class T>
__global__ void __launch_bounds__(64, 14) k_lbm_far_pairs(const T *__restrict__ fin, T *__restrict__ fout, LbmParams p,
                                                      const unsigned *__restrict__ bits,
                                                      const unsigned *__restrict__ seed_in) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    if (region_has(bits, tile_index(p, x0 >> p.tlx, y >> p.tly, z >> p.tlz))) return;
    const unsigned seed = *seed_in;
    if (y > 0 && y < p.ny - 1)
        lbm_pair<T, false, false>(fin, fout, nullptr, p, x0, y, z, nullptr, seed);
    else
        lbm_pair<T, true, false>(fin, fout, nullptr, p, x0, y, z, nullptr, seed);
}

template <class T>
__global__ void __launch_bounds__(64) k_lbm_near_pairs(const T *__restrict__ fin, T *__restrict__ fout,
                                                       float4 *__restrict__ F, LbmParams p,
                                                       const unsigned *__restrict__ bits, float4 *__restrict__ vel,
                                                       const unsigned *__restrict__ seed_in,
                                                       unsigned *__restrict__ seed_out) {
    const unsigned seed = *seed_in;
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *seed_out = seed + 1u;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= p.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    if (!region_has(bits, tile_index(p, x0 >> p.tlx, y >> p.tly, z >> p.tlz))) return;
    if (y > 0 && y < p.ny - 1)
        lbm_pair<T, false, true>(fin, fout, F, p, x0, y, z, vel, seed);
    else
        lbm_pair<T, true, true>(fin, fout, F, p, x0, y, z, vel, seed);
}

// Grid of the pair kernels: up to 64 pairs per block along x.
static dim3 pair_grid(const LbmParams &p, int &bx) {
    const int pairs = p.nx / 2;
    bx = pairs < 64 ? pairs : 64;
    return dim3((pairs + bx - 1) / bx, p.ny, p.nz);
}

// The pair form applies to 16-bit storage with nx even, when the launch
// shape asks for it.
template <class T>
static bool use_pairs(const LbmParams &p) {
    return sizeof(T) == 2 && p.pairs && p.nx % 2 == 0;
}

// rho and u(t) on every node after a step. On the last step's force region
// (bits; null: none) u(t) is the value the near field stored (vel): the force
// field there has been consumed. Elsewhere it follows from the post-collision
// populations and the force of the same step: rho = 1 + sum d*_q,
// rho u = sum c_q d*_q - F/2 (the collision adds exactly F to the momentum,
// and rho u = sum c_q d_q + F/2 before it).
template <class T>
__global__ void k_macro(const T *__restrict__ f, const float4 *__restrict__ F, LbmParams p,
                        const unsigned *__restrict__ bits, const float4 *__restrict__ vel, double *rho, double *u) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = p.N;  // 64-bit population offsets q * N + n
    if (n >= N) return;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const float d = Pop<T>::ld(f + q * N + n) * pop_unscale<T>(q);
        drho += d;
        if (cx(q)) jx += cx(q) * d;
        if (cy(q)) jy += cy(q) * d;
        if (cz(q)) jz += cz(q) * d;
    }
    const float r = 1.f + drho;
    if (rho) rho[n] = (double)r;
    if (!u) return;
    const int x = n % p.nx, y = (n / p.nx) % p.ny, z = n / (p.nx * p.ny);
    float ux, uy, uz;
    if (bits && region_has(bits, tile_index(p, x >> p.tlx, y >> p.tly, z >> p.tlz))) {
        const float4 q = vel[n];
        ux = q.x;
        uy = q.y;
        uz = q.z;
    } else {
        bool nonzero;
        const float4 a = force_at(F, p, n, nonzero);
        const float Fx = a.x + p.gx, Fy = a.y + p.gy, Fz = a.z + p.gz;
        ux = (jx - 0.5f * Fx) / r;
        uy = (jy - 0.5f * Fy) / r;
        uz = (jz - 0.5f * Fz) / r;
    }
    u[3 * (size_t)n + 0] = (double)ux;
    u[3 * (size_t)n + 1] = (double)uy;
    u[3 * (size_t)n + 2] = (double)uz;
}

// ---------------------------------------------------------------- launchers
size_t pop_bytes(int fmt) { return fmt == POP_F32 ? 4 : 2; }

template <class T>
static cudaError_t lbm_t(const void *fin, void *fout, const LbmParams &p, const unsigned *seed, unsigned *next_seed,
                         cudaStream_t s) {
    if constexpr (sizeof(T) == 2) {
        if (use_pairs<T>(p)) {
            int bx;
            const dim3 grid = pair_grid(p, bx);
            k_lbm_pairs<T><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p, seed, next_seed);
            return cudaGetLastError();
        }
    }
    const int bx = p.nx < 128 ? p.nx : 128;
    dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
    k_lbm<T><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p, seed, next_seed);
    return cudaGetLastError();
}

template <class T>
static cudaError_t far_t(const void *fin, void *fout, const LbmParams &p, const unsigned *bits, const unsigned *seed,
                         bool spec, cudaStream_t s) {
    if constexpr (sizeof(T) == 2) {
        if (use_pairs<T>(p)) {
            int bx;
            const dim3 grid = pair_grid(p, bx);
            k_lbm_far_pairs<T><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p, bits, seed);
            return cudaGetLastError();
        }
    }
    const int bx = p.nx < 128 ? p.nx : 128;
    dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
    if constexpr (std::is_same<T, float>::value) {
        if (p.l2) {  // L2-normal form (FP32 only)
            if (spec)
                k_lbm_far<T, true, false><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p,
                                                              bits, seed);
            else
                k_lbm_far<T, false, false><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p,
                                                               bits, seed);
            return cudaGetLastError();
        }
    }
    if (spec)
        k_lbm_far<T, true><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p, bits, seed);
    else
        k_lbm_far<T, false><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), p, bits, seed);
    return cudaGetLastError();
}

template <class T>
static cudaError_t near_t(const void *fin, void *fout, float4 *F, const LbmParams &p, const unsigned *bits,
                          float4 *vel, int blocks, const unsigned *seed, unsigned *next_seed, cudaStream_t s) {
    const int nwords = (int)(((long long)p.ntx * p.nty * p.ntz + 31) / 32);
    const size_t smem = sizeof(int) * ((size_t)nwords + 1);
    if constexpr (std::is_same<T, float>::value) {
        if (p.l2) {  // L2-normal form (FP32 only)
            if (blocks <= 0) {
                const int bx = p.nx < 128 ? p.nx : 128;
                dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
                k_lbm_near_rows<T, false><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), F, p,
                                                              bits, vel, seed, next_seed);
            } else {
                k_lbm_near<T, false><<<blocks, kTileBlock, smem, s>>>(static_cast<const T *>(fin),
                                                                      static_cast<T *>(fout), F, p, bits, nwords, vel,
                                                                      seed, next_seed);
            }
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(T) == 2) {
        if (blocks <= 0 && use_pairs<T>(p)) {  // rows over the whole lattice, two nodes per thread
            int bx;
            const dim3 grid = pair_grid(p, bx);
            k_lbm_near_pairs<T><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), F, p, bits,
                                                     vel, seed, next_seed);
            return cudaGetLastError();
        }
    }
    if (blocks <= 0) {  // rows over the whole lattice
        const int bx = p.nx < 128 ? p.nx : 128;
        dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
        k_lbm_near_rows<T><<<grid, bx, 0, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), F, p, bits, vel,
                                               seed, next_seed);
        return cudaGetLastError();
    }
    k_lbm_near<T><<<blocks, kTileBlock, smem, s>>>(static_cast<const T *>(fin), static_cast<T *>(fout), F, p, bits,
                                                   nwords, vel, seed, next_seed);
    return cudaGetLastError();
}

// Every list-form near-field kernel may take up to 4 (max_words + 1) bytes
// of dynamic shared memory.
cudaError_t prepare_near_field(long long max_words) {
    const int smem = (int)(sizeof(int) * (max_words + 1));
    if (smem <= 48 * 1024) return cudaSuccess;
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_lbm_near<float, true>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lbm_near<float, false>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lbm_near<__half, true>, a, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lbm_near<__nv_bfloat16, true>, a, smem);
    return e;
}

bool is_lbm_far_kernel(const void *fn) {
    return fn == (const void *)k_lbm_far_pairs<__half> || fn == (const void *)k_lbm_far_pairs<__nv_bfloat16> ||
           fn == (const void *)k_lbm_far<float, false, false> || fn == (const void *)k_lbm_far<float, true, false> ||
           fn == (const void *)k_lbm_far<float, false> || fn == (const void *)k_lbm_far<__half, false> ||
           fn == (const void *)k_lbm_far<__nv_bfloat16, false> || fn == (const void *)k_lbm_far<float, true> ||
           fn == (const void *)k_lbm_far<__half, true> || fn == (const void *)k_lbm_far<__nv_bfloat16, true>;
}

cudaError_t launch_lbm(const void *fin, void *fout, const LbmParams &p, const unsigned *seed, unsigned *next_seed,
                       cudaStream_t s) {
    switch (p.fmt) {
        case POP_F16: return lbm_t<__half>(fin, fout, p, seed, next_seed, s);
        case POP_BF16: return lbm_t<__nv_bfloat16>(fin, fout, p, seed, next_seed, s);
        default: return lbm_t<float>(fin, fout, p, seed, next_seed, s);
    }
}

cudaError_t launch_lbm_far(const void *fin, void *fout, const LbmParams &p, const unsigned *bits,
                           const unsigned *seed, bool spec, cudaStream_t s) {
    switch (p.fmt) {
        case POP_F16: return far_t<__half>(fin, fout, p, bits, seed, spec, s);
        case POP_BF16: return far_t<__nv_bfloat16>(fin, fout, p, bits, seed, spec, s);
        default: return far_t<float>(fin, fout, p, bits, seed, spec, s);
    }
}

cudaError_t launch_lbm_near(const void *fin, void *fout, float4 *F, const LbmParams &p, const unsigned *bits,
                            float4 *vel, int blocks, const unsigned *seed, unsigned *next_seed, cudaStream_t s) {
    switch (p.fmt) {
        case POP_F16: return near_t<__half>(fin, fout, F, p, bits, vel, blocks, seed, next_seed, s);
        case POP_BF16: return near_t<__nv_bfloat16>(fin, fout, F, p, bits, vel, blocks, seed, next_seed, s);
        default: return near_t<float>(fin, fout, F, p, bits, vel, blocks, seed, next_seed, s);
    }
}

cudaError_t launch_lbm_init(void *f, const LbmParams &p, cudaStream_t s) {
    // rest equilibrium, rho = 1, u = 0: every deviation is zero (all-zero bits
    // in every storage format)
    return cudaMemsetAsync(f, 0, pop_bytes(p.fmt) * 19 * (size_t)p.N, s);
}

cudaError_t launch_lbm_macro(const void *f, const float4 *F, const LbmParams &p, const unsigned *bits,
                             const float4 *vel, double *rho, double *u, cudaStream_t s) {
    const int blocks = (int)((p.N + 255) / 256);
    switch (p.fmt) {
        case POP_F16:
            k_macro<__half><<<blocks, 256, 0, s>>>(static_cast<const __half *>(f), F, p, bits, vel, rho, u);
            break;
        case POP_BF16:
            k_macro<__nv_bfloat16>
                <<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(f), F, p, bits, vel, rho, u);
            break;
        default: k_macro<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(f), F, p, bits, vel, rho, u);
    }
    return cudaGetLastError();
}

}  // namespace cf
