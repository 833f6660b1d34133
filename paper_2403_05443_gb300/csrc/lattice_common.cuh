// Device code shared by the lattice kernels: storage policies for the
// distribution deviations and the BGK collision with Guo forcing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbsph_internal.cuh"

namespace lbsph {

// ---------------------------------------------------------------------------
// storage policies: values are deviations f_i - w_i rho0 (x scale for FP16)
struct StF32 {
    using T = float;
    static __device__ __forceinline__ float4 ld4(const T* p, float) { return __ldg(reinterpret_cast<const float4*>(p)); }
    static __device__ __forceinline__ float ld1(const T* p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st4(T* p, float4 v, float) { *reinterpret_cast<float4*>(p) = v; }
    static __device__ __forceinline__ void st1(T* p, float v, float) { *p = v; }
};

struct StF16 {
    using T = __half;
    static __device__ __forceinline__ float4 ld4(const T* p, float inv)
    {
        uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x * inv, a.y * inv, b.x * inv, b.y * inv);
    }
    static __device__ __forceinline__ float ld1(const T* p, float inv) { return __half2float(p[0]) * inv; }
    static __device__ __forceinline__ void st4(T* p, float4 v, float scale)
    {
        __half2 a = __floats2half2_rn(v.x * scale, v.y * scale);
        __half2 b = __floats2half2_rn(v.z * scale, v.w * scale);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = u;
    }
    static __device__ __forceinline__ void st1(T* p, float v, float scale) { *p = __float2half_rn(v * scale); }
};

struct StBF16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float4 ld4(const T* p, float)
    {
        uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float ld1(const T* p, float) { return __bfloat162float(p[0]); }
    static __device__ __forceinline__ void st4(T* p, float4 v, float)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = u;
    }
    static __device__ __forceinline__ void st1(T* p, float v, float) { *p = __float2bfloat16_rn(v); }
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

// BGK collision (Eq. 3-4) on deviations with Guo forcing; eps is the mass put
// back by an earlier remap (w_i eps added to every population first).
__device__ __forceinline__ void collide19(float (&f)[Q], float omega, float rho0, float gx, float gy,
                                          float gz, float eps)
{
    if (eps != 0.0f) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] += w_of(i) * eps;
    }
    float drho = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) drho += f[i];
    const float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    const float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    const float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
    const float rho = rho0 + drho;
    const float ir = 1.0f / rho;
    const float ux = (jx + 0.5f * gx) * ir, uy = (jy + 0.5f * gy) * ir, uz = (jz + 0.5f * gz) * ir;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float ug = ux * gx + uy * gy + uz * gz;
    const float om1 = 1.0f - omega;
    const float cf = 1.0f - 0.5f * omega;
    {
        const float w = w_of(0);
        f[0] = om1 * f[0] + omega * w * (drho - 1.5f * rho * uu) - 3.0f * cf * w * ug;
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
        const float cg = cx_of(i) * gx + cy_of(i) * gy + cz_of(i) * gz;
        const float w = w_of(i);
        const float sym = w * (drho + rho * (4.5f * cu * cu - 1.5f * uu));
        const float asym = 3.0f * w * rho * cu;
        const float ss = cf * w * (9.0f * cu * cg - 3.0f * ug);
        const float sa = 3.0f * cf * w * cg;
        const float a = f[i], b = f[i + 1];
        f[i] = om1 * a + omega * (sym + asym) + ss + sa;
        f[i + 1] = om1 * b + omega * (sym - asym) + ss - sa;
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
