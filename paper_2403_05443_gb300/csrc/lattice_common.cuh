// Device code shared by the lattice kernels: storage policies for the
// distribution deviations and the BGK collision with Guo forcing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbsph_internal.cuh"

namespace lbsph {

// ---------------------------------------------------------------------------
// Loads of data that another block may have written earlier in the same
// (persistent) kernel go through L2 (ld.global.cg): the SM's L1 is not
// coherent and could still hold a line from an earlier step.
__device__ __forceinline__ BoxDyn ldcg_dyn(const BoxDyn* p)
{
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    BoxDyn d;
    d.g[0] = v.x; d.g[1] = v.y; d.g[2] = v.z; d.eps = v.w;
    return d;
}
__device__ __forceinline__ NeedHdr ldcg_hdr(const NeedHdr* p)
{
    const int4 v = __ldcg(reinterpret_cast<const int4*>(p));
    NeedHdr h;
    h.ow[0] = v.x; h.ow[1] = v.y; h.ow[2] = v.z; h.S = v.w;
    return h;
}
// block-wide copy of a struct from global to shared memory, 4-byte words
template <class T>
__device__ __forceinline__ void ldcg_copy(T* dst, const T* src, int tid, int nthreads)
{
    static_assert(sizeof(T) % 4 == 0, "copied as 4-byte words");
    const unsigned* s = reinterpret_cast<const unsigned*>(src);
    unsigned* d = reinterpret_cast<unsigned*>(dst);
    for (int j = tid; j < (int)(sizeof(T) / 4); j += nthreads) d[j] = __ldcg(s + j);
}

// ---------------------------------------------------------------------------
// L2 eviction priority of lattice accesses.  The bulk streams twice the size
// of L2 per step; with evict-first on its traffic, the particle chain's state
// and the lattice around the particles stay in L2.  Lattice loads never
// allocate in L1 (the L1 is not coherent across the steps of a persistent
// kernel).
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_evict_normal()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float4 ldh_f4(const void* a, unsigned long long pol)
{
    float4 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldh_f1(const void* a, unsigned long long pol)
{
    float v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ldh_u2(const void* a, unsigned long long pol)
{
    uint2 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned short ldh_u16(const void* a, unsigned long long pol)
{
    unsigned short v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void sth_f4(void* a, float4 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void sth_f1(void* a, float v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void sth_u2(void* a, uint2 v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1,%2}, %3;" ::"l"(a), "r"(v.x), "r"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void sth_u16(void* a, unsigned short v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(a), "h"(v), "l"(pol) : "memory");
}

// ---------------------------------------------------------------------------
// storage policies: values are deviations f_i - w_i rho0 (x scale for FP16).
// ld4/ld1/st4/st1 convert to and from physical units; the raw forms keep the
// stored scale (SCALED: FP16), for the bulk tile, whose collision works in
// stored units (ColliderT<true>).
struct StF32 {
    using T = float;
    static constexpr bool SCALED = false;
    static constexpr bool GHOST = false;       // collision: BGK
    static __device__ __forceinline__ float4 ld4(const T* p, float, unsigned long long pol) { return ldh_f4(p, pol); }
    static __device__ __forceinline__ float ld1(const T* p, float, unsigned long long pol) { return ldh_f1(p, pol); }
    static __device__ __forceinline__ void st4(T* p, float4 v, float, unsigned long long pol) { sth_f4(p, v, pol); }
    static __device__ __forceinline__ void st1(T* p, float v, float, unsigned long long pol) { sth_f1(p, v, pol); }
    static __device__ __forceinline__ float4 ld4r(const T* p, unsigned long long pol) { return ldh_f4(p, pol); }
    static __device__ __forceinline__ float ld1r(const T* p, unsigned long long pol) { return ldh_f1(p, pol); }
    static __device__ __forceinline__ void st4r(T* p, float4 v, unsigned long long pol) { sth_f4(p, v, pol); }
    static __device__ __forceinline__ void st1r(T* p, float v, unsigned long long pol) { sth_f1(p, v, pol); }
};

struct StF16 {
    using T = __half;
    static constexpr bool SCALED = true;
    static constexpr bool GHOST = false;
    static __device__ __forceinline__ float4 ld4(const T* p, float inv, unsigned long long pol)
    {
        const uint2 u = ldh_u2(p, pol);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x * inv, a.y * inv, b.x * inv, b.y * inv);
    }
    static __device__ __forceinline__ float ld1(const T* p, float inv, unsigned long long pol)
    {
        return __half2float(__ushort_as_half(ldh_u16(p, pol))) * inv;
    }
    static __device__ __forceinline__ void st4(T* p, float4 v, float scale, unsigned long long pol)
    {
        __half2 a = __floats2half2_rn(v.x * scale, v.y * scale);
        __half2 b = __floats2half2_rn(v.z * scale, v.w * scale);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        sth_u2(p, u, pol);
    }
    static __device__ __forceinline__ void st1(T* p, float v, float scale, unsigned long long pol)
    {
        sth_u16(p, __half_as_ushort(__float2half_rn(v * scale)), pol);
    }
    static __device__ __forceinline__ float4 ld4r(const T* p, unsigned long long pol)
    {
        const uint2 u = ldh_u2(p, pol);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float ld1r(const T* p, unsigned long long pol)
    {
        return __half2float(__ushort_as_half(ldh_u16(p, pol)));
    }
    static __device__ __forceinline__ void st4r(T* p, float4 v, unsigned long long pol)
    {
        __half2 a = __floats2half2_rn(v.x, v.y);
        __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        sth_u2(p, u, pol);
    }
    static __device__ __forceinline__ void st1r(T* p, float v, unsigned long long pol)
    {
        sth_u16(p, __half_as_ushort(__float2half_rn(v)), pol);
    }
};

struct StBF16 {
    using T = __nv_bfloat16;
    static constexpr bool SCALED = false;
    static constexpr bool GHOST = false;
    static __device__ __forceinline__ float4 ld4(const T* p, float, unsigned long long pol)
    {
        const uint2 u = ldh_u2(p, pol);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float ld1(const T* p, float, unsigned long long pol)
    {
        return __bfloat162float(__ushort_as_bfloat16(ldh_u16(p, pol)));
    }
    static __device__ __forceinline__ void st4(T* p, float4 v, float, unsigned long long pol)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        sth_u2(p, u, pol);
    }
    static __device__ __forceinline__ void st1(T* p, float v, float, unsigned long long pol)
    {
        sth_u16(p, __bfloat16_as_ushort(__float2bfloat16_rn(v)), pol);
    }
    static __device__ __forceinline__ float4 ld4r(const T* p, unsigned long long pol) { return ld4(p, 1.0f, pol); }
    static __device__ __forceinline__ float ld1r(const T* p, unsigned long long pol) { return ld1(p, 1.0f, pol); }
    static __device__ __forceinline__ void st4r(T* p, float4 v, unsigned long long pol) { st4(p, v, 1.0f, pol); }
    static __device__ __forceinline__ void st1r(T* p, float v, unsigned long long pol) { st1(p, v, 1.0f, pol); }
};

// FP32 storage with the paper's collision (ghost modes relaxed at once, see
// ColliderT): the same layout as StF32.
struct StF32G : StF32 {
    static constexpr bool GHOST = true;
};

// ---------------------------------------------------------------------------
__device__ __forceinline__ float comp(const float4& v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_comp(float4& v, int k, float a)
{
    if (k == 0) v.x = a; else if (k == 1) v.y = a; else if (k == 2) v.z = a; else v.w = a;
}

// BGK collision (Eq. 3-4) on deviations d_i = f_i - w_i rho0 with Guo
// forcing, arranged per pair of opposite directions (i, i+1 for odd i).  With
// rho = rho0 + sum d, j = sum c d, u = (j + g/2)/rho and cf = 1 - omega/2, the
// post-collision deviations are
//   d_i' = (1 - omega) d_i + sym_i + asym_i,  d_{i+1}' = (1 - omega) d_{i+1} + sym_i - asym_i,
//   sym_i  = w_i P + cu (4.5 omega rho w_i cu + 9 cf w_i (c_i.g)),
//   asym_i = 3 omega rho w_i cu + 3 cf w_i (c_i.g),
//   P = omega drho - 1.5 omega rho u.u - 3 cf u.g  (+ (1 - omega) eps),
// cu = c_i.u; the rest population gets d_0' = (1 - omega) d_0 + w_0 P.  This is
// the BGK relaxation to the second-order equilibrium plus (1 - omega/2) times
// the Guo source w_i [3 (c_i - u).g + 9 (c_i.u)(c_i.g)], with every term that
// depends only on the box's uniform force g computed once per box.  eps is the
// mass put back by an earlier remap: w_i eps is added to every population
// first, which only moves drho and P.
//
// SCALED: the populations come and go in stored units (times the FP16 storage
// scale sc, a power of two): drho and j are brought to physical units by one
// multiplication each, and omega (where it multiplies an equilibrium term),
// 3 cf, eps and the force terms are held times sc, so that P and the pair terms
// come out times sc; no population is scaled on load or on store.  With a
// power-of-two sc each of these products is exact, so the results are the
// same bits as scaling every population.
//
// GHOST (FP32 only): the collision the paper's simulations use (Sec. II.A: one
// relaxation time for the non-conserved hydrodynamic modes, the
// non-hydrodynamic ("ghost") modes relaxed at once to equilibrium).  Of the
// non-equilibrium part only its projection on the hydrodynamic Hermite modes
// is kept and relaxed:
//   d_i' = deq_i + (1 - omega) w_i [3 c_i.j_neq + 4.5 (c_i c_i - I/3) : Pi_neq] + S_i,
// deq_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)), S_i the Guo source,
// j_neq = j - rho u = -g/2, Pi_neq = sum_i c_i c_i d_i + (eps - drho)/3 I - rho u u
// (the mass return eps added to every population first, as above).  Per pair
// the odd part is 3 w rho cu + 1.5 w (c_i.g) whatever omega (the momentum
// gains g), the even part w (drho + rho (4.5 cu^2 - 1.5 u.u)) + (1 - omega)
// 4.5 w Q_i + cf w (9 cu (c_i.g) - 3 u.g), Q_i = c_i.Pi_neq.c_i - tr Pi_neq / 3.
// At omega = 1 it is BGK.
template <bool SCALED, bool GHOST = false>
struct ColliderT {
    static_assert(!(SCALED && GHOST), "the ghost-mode collision works on unscaled populations");
    float omega, om1, rho0, eps;    // SCALED: omega and eps times sc
    float gx, gy, gz;
    float cfug;                     // 3 cf, the factor of u.g in P (times sc)
    float l[9];                     // per pair: 3 cf w (c.g) (times sc); 9 cf w (c.g) is 3 l
    float isc;                      // SCALED: 1 / sc

    __device__ __forceinline__ void init(float omega_, float rho0_, float gx_, float gy_, float gz_, float eps_,
                                         float scale = 1.0f, float inv_scale = 1.0f)
    {
        const float s = SCALED ? scale : 1.0f;
        omega = omega_ * s;
        om1 = 1.0f - omega_;
        rho0 = rho0_;
        eps = eps_ * s;
        gx = gx_; gy = gy_; gz = gz_;
        isc = inv_scale;
        const float cf = 1.0f - 0.5f * omega_;
        cfug = (3.0f * cf) * s;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            const float cg = cx_of(i) * gx_ + cy_of(i) * gy_ + cz_of(i) * gz_;
            l[m] = ((3.0f * w_of(i)) * cf * cg) * s;
        }
    }

    __device__ __forceinline__ void apply(float (&f)[Q]) const
    {
        if constexpr (GHOST) {
            apply_ghost(f);
        } else {
            apply_bgk(f);
        }
    }

    __device__ __forceinline__ void apply_bgk(float (&f)[Q]) const
    {
        float sm[9], df[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            sm[m] = f[2 * m + 1] + f[2 * m + 2];
            df[m] = f[2 * m + 1] - f[2 * m + 2];
        }
        float drho = f[0] + eps;
#pragma unroll
        for (int m = 0; m < 9; ++m) drho += sm[m];
        float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            if (cx_of(i) == 1) jx += df[m]; else if (cx_of(i) == -1) jx -= df[m];
            if (cy_of(i) == 1) jy += df[m]; else if (cy_of(i) == -1) jy -= df[m];
            if (cz_of(i) == 1) jz += df[m]; else if (cz_of(i) == -1) jz -= df[m];
        }
        if (SCALED) {
            drho *= isc;
            jx *= isc;
            jy *= isc;
            jz *= isc;
        }
        const float rho = rho0 + drho;
        const float ir = __fdividef(1.0f, rho);
        const float ux = (jx + 0.5f * gx) * ir, uy = (jy + 0.5f * gy) * ir, uz = (jz + 0.5f * gz) * ir;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float ug = ux * gx + uy * gy + uz * gz;
        const float orho = omega * rho;
        const float P = omega * drho - 1.5f * orho * uu - cfug * ug + om1 * eps;
        f[0] = om1 * f[0] + w_of(0) * P;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            const float w = w_of(i);
            const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
            const float sym = w * P + cu * ((4.5f * w) * orho * cu + 3.0f * l[m]);
            const float asym = (3.0f * w) * orho * cu + l[m];
            f[i] = om1 * f[i] + (sym + asym);
            f[i + 1] = om1 * f[i + 1] + (sym - asym);
        }
    }

    __device__ __forceinline__ void apply_ghost(float (&f)[Q]) const
    {
        float sm[9], df[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            sm[m] = f[2 * m + 1] + f[2 * m + 2];
            df[m] = f[2 * m + 1] - f[2 * m + 2];
        }
        float drho = f[0] + eps;
#pragma unroll
        for (int m = 0; m < 9; ++m) drho += sm[m];
        float jx = 0.0f, jy = 0.0f, jz = 0.0f;
        float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
            if (cx == 1) jx += df[m]; else if (cx == -1) jx -= df[m];
            if (cy == 1) jy += df[m]; else if (cy == -1) jy -= df[m];
            if (cz == 1) jz += df[m]; else if (cz == -1) jz -= df[m];
            if (cx) pxx += sm[m];
            if (cy) pyy += sm[m];
            if (cz) pzz += sm[m];
            if (cx * cy == 1) pxy += sm[m]; else if (cx * cy == -1) pxy -= sm[m];
            if (cx * cz == 1) pxz += sm[m]; else if (cx * cz == -1) pxz -= sm[m];
            if (cy * cz == 1) pyz += sm[m]; else if (cy * cz == -1) pyz -= sm[m];
        }
        const float rho = rho0 + drho;
        const float ir = __fdividef(1.0f, rho);
        const float ux = (jx + 0.5f * gx) * ir, uy = (jy + 0.5f * gy) * ir, uz = (jz + 0.5f * gz) * ir;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float ug = ux * gx + uy * gy + uz * gz;
        // Pi_neq (the populations' second moment beyond the rest state w rho0
        // is sum c c d + eps/3 I; that of the equilibrium rho/3 I + rho u u)
        const float iso = (eps - drho) * (1.0f / 3.0f);
        const float nxx = pxx + iso - rho * ux * ux, nyy = pyy + iso - rho * uy * uy, nzz = pzz + iso - rho * uz * uz;
        const float nxy = pxy - rho * ux * uy, nxz = pxz - rho * ux * uz, nyz = pyz - rho * uy * uz;
        const float tr3 = (nxx + nyy + nzz) * (1.0f / 3.0f);
        const float cf = 1.0f - 0.5f * omega;
        const float even0 = drho - 1.5f * rho * uu - 3.0f * cf * ug;   // times w: the even part's common terms
        f[0] = w_of(0) * (even0 - om1 * 4.5f * tr3);
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
            const float w = w_of(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cg = cx * gx + cy * gy + cz * gz;
            float qn = -tr3;
            if (cx) qn += nxx;
            if (cy) qn += nyy;
            if (cz) qn += nzz;
            if (cx * cy) qn += 2.0f * (cx * cy) * nxy;
            if (cx * cz) qn += 2.0f * (cx * cz) * nxz;
            if (cy * cz) qn += 2.0f * (cy * cz) * nyz;
            const float sym = w * (even0 + 4.5f * rho * cu * cu + om1 * 4.5f * qn + 9.0f * cf * cu * cg);
            const float asym = w * (3.0f * rho * cu + 1.5f * cg);
            f[i] = sym + asym;
            f[i + 1] = sym - asym;
        }
    }
};

using Collider = ColliderT<false>;

// one node's collision with freshly set-up box terms
template <bool GHOST = false>
__device__ __forceinline__ void collide19(float (&f)[Q], float omega, float rho0, float gx, float gy,
                                          float gz, float eps)
{
    ColliderT<false, GHOST> C;
    C.init(omega, rho0, gx, gy, gz, eps);
    C.apply(f);
}


// The collision of one node, split between two threads: half H = 0 updates the
// rest population and the pairs of directions 1..10, H = 1 the pairs 11..18,
// both from the node's totals t = (sum d, j, and for GHOST the second moments
// sum c c d), which both halves hold bit for bit.  The formulas are those of
// ColliderT (unscaled populations), with the same eps convention: w_i eps is
// added to every population first.
template <bool GHOST, int H, int NT>
__device__ __forceinline__ void collide_half(float (&f)[Q], const float (&t)[NT], float omega, float rho0,
                                             float gx, float gy, float gz, float eps)
{
    const float om1 = 1.0f - omega, cf = 1.0f - 0.5f * omega;
    const float drho = t[0] + eps;
    const float rho = rho0 + drho;
    const float ir = __fdividef(1.0f, rho);
    const float ux = (t[1] + 0.5f * gx) * ir, uy = (t[2] + 0.5f * gy) * ir, uz = (t[3] + 0.5f * gz) * ir;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float ug = ux * gx + uy * gy + uz * gz;
    if constexpr (!GHOST) {
        const float orho = omega * rho;
        const float Pc = omega * drho - 1.5f * orho * uu - 3.0f * cf * ug + om1 * eps;
        if (H == 0) f[0] = om1 * f[0] + w_of(0) * Pc;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            if (H == 0 ? i > 10 : i < 11) continue;
            const float w = w_of(i);
            const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
            const float l = (3.0f * w) * cf * (cx_of(i) * gx + cy_of(i) * gy + cz_of(i) * gz);
            const float sym = w * Pc + cu * ((4.5f * w) * orho * cu + 3.0f * l);
            const float asym = (3.0f * w) * orho * cu + l;
            f[i] = om1 * f[i] + (sym + asym);
            f[i + 1] = om1 * f[i + 1] + (sym - asym);
        }
    } else {
        static_assert(NT >= 10, "the ghost-mode collision needs the second moments");
        const float iso = (eps - drho) * (1.0f / 3.0f);
        const float nxx = t[4] + iso - rho * ux * ux, nyy = t[5] + iso - rho * uy * uy, nzz = t[6] + iso - rho * uz * uz;
        const float nxy = t[7] - rho * ux * uy, nxz = t[8] - rho * ux * uz, nyz = t[9] - rho * uy * uz;
        const float tr3 = (nxx + nyy + nzz) * (1.0f / 3.0f);
        const float even0 = drho - 1.5f * rho * uu - 3.0f * cf * ug;
        if (H == 0) f[0] = w_of(0) * (even0 - om1 * 4.5f * tr3);
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int i = 2 * m + 1;
            if (H == 0 ? i > 10 : i < 11) continue;
            const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
            const float w = w_of(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cg = cx * gx + cy * gy + cz * gz;
            float qn = -tr3;
            if (cx) qn += nxx;
            if (cy) qn += nyy;
            if (cz) qn += nzz;
            if (cx * cy) qn += 2.0f * (cx * cy) * nxy;
            if (cx * cz) qn += 2.0f * (cx * cz) * nxz;
            if (cy * cz) qn += 2.0f * (cy * cz) * nyz;
            const float sym = w * (even0 + 4.5f * rho * cu * cu + om1 * 4.5f * qn + 9.0f * cf * cu * cg);
            const float asym = w * (3.0f * rho * cu + 1.5f * cg);
            f[i] = sym + asym;
            f[i + 1] = sym - asym;
        }
    }
}

__device__ __forceinline__ long long fixp(float v) { return __float2ll_rn(v * FIXF); }

__device__ __forceinline__ int wrapd(int m, int L) { return m < 0 ? m + L : (m >= L ? m - L : m); }

// Squirmer slip of Eq. squirmer at r = x_b - x_c for a spheroid with long axis
// e, semi-axis a, eccentricity^2 eps2 and modes B1, B2, in FP32.
__device__ __forceinline__ void squirmer_slip(const float e[3], float a, float eps2, float B1, float B2, float rx,
                                              float ry, float rz, float& sx, float& sy, float& sz)
{
    const float zr = rx * e[0] + ry * e[1] + rz * e[2];
    const float px = rx - zr * e[0], py = ry - zr * e[1], pz = rz - zr * e[2];
    const float rho = sqrtf(px * px + py * py + pz * pz);
    sx = sy = sz = 0.0f;
    if (rho < 1e-5f) return;
    const float z = fminf(fmaxf(zr, -a), a);
    const float den = sqrtf(a * a - eps2 * z * z);
    const float se = -sqrtf(fmaxf(a * a - z * z, 0.0f)) / den;
    const float sp = sqrtf(1.0f - eps2) * z / den;
    const float eps = sqrtf(eps2);
    float zeta;
    if (eps < 1e-4f) {
        zeta = zr / a;
    } else {
        const float d1 = sqrtf(rho * rho + (zr + a * eps) * (zr + a * eps));
        const float d2 = sqrtf(rho * rho + (zr - a * eps) * (zr - a * eps));
        zeta = (d1 - d2) / (2.0f * a * eps);
    }
    const float amp = -(B1 + B2 * zeta) * se;
    const float ir = 1.0f / rho;
    sx = amp * (se * e[0] + sp * px * ir);
    sy = amp * (se * e[1] + sp * py * ir);
    sz = amp * (se * e[2] + sp * pz * ir);
}

}  // namespace lbsph
