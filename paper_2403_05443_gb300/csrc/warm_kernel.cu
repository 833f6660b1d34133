// Warm start of a run (lb_init_fluid, lb_stokes_field): an initial fluid at
// the local equilibrium of a given velocity field, and the periodic Stokes flow
// driven by the particles' external forces, as that field.
//
// Stokes flow (mu Lap u - grad p + g = 0, div u = 0 on the periodic lattice):
// the force density g puts F_ext of each particle uniformly on its solid nodes
// and the box's uniform counter force and body force on the fluid nodes; the
// mean of g (if the forces do not balance) is dropped.  In Fourier space, with
// kt_d = 2 sin(pi k_d / n_d) (the symbol of the nearest-neighbour difference,
// so that |kt|^2 is the symbol of the 7-point Laplacian),
//   u^(k) = (g^ - kt (kt . g^) / |kt|^2) / (mu |kt|^2),  u^(0) = 0.
// The transforms are separable DFTs along x, y and z computed by definition,
// one output element per thread with the line's twiddle table in shared
// memory (box edges are not powers of two in general); FP32 complex.
#include "lattice_common.cuh"

namespace lbsph {

// f = f_eq(rho0, u) - w rho0 on fluid nodes (deviation storage), 0 elsewhere
template <class St>
__global__ void init_fluid_kernel(const BoxDev B, void* fbuf, const float* u, const int* owner)
{
    using T = typename St::T;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= B.N) return;
    T* f = reinterpret_cast<T*>(fbuf) + B.off;
    const bool fluid = owner[n] == 0;
    const float ux = fluid ? u[n] : 0.0f, uy = fluid ? u[B.N + n] : 0.0f, uz = fluid ? u[2 * B.N + n] : 0.0f;
    const float uu = ux * ux + uy * uy + uz * uz;
    const unsigned long long pol = l2_evict_normal();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
        const float d = fluid ? w_of(i) * B.rho0f * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu) : 0.0f;
        St::st1(f + (long long)i * B.N + n, d, B.scale, pol);
    }
}

// solid-node count of each particle of the box (owner = p + 1) and fluid count
__global__ void count_owner_kernel(const int* owner, long long N, int* counts, int np)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int o = owner[n];
    if (o > 0 && o <= np) atomicAdd(counts + o, 1);
    else if (o == 0) atomicAdd(counts, 1);
}

// force density as complex [3][N]: F_ext / nsolid on a particle's solid nodes,
// the body force plus (counter_on) -sum F_ext / N_fluid on fluid nodes
__global__ void force_density_kernel(const int* owner, long long N, const int* counts, const PartDev* pd, int np,
                                     int counter_on, double bx, double by, double bz, float2* g)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int o = owner[n];
    double f[3] = {0.0, 0.0, 0.0};
    if (o > 0 && o <= np) {
        const double c = 1.0 / (double)counts[o];
        for (int k = 0; k < 3; ++k) f[k] = pd[o - 1].Fext[k] * c;
    } else if (o == 0) {
        f[0] = bx; f[1] = by; f[2] = bz;
        if (counter_on && counts[0] > 0) {
            for (int p = 0; p < np; ++p)
                for (int k = 0; k < 3; ++k) f[k] -= pd[p].Fext[k] / (double)counts[0];
        }
    }
    for (int k = 0; k < 3; ++k) g[k * N + n] = make_float2((float)f[k], 0.0f);
}

// one DFT pass along one axis: out(.., k, ..) = sum_j in(.., j, ..) w^(j k),
// w = exp(sign 2 pi i / n); three components of [nz][ny][nx] each
__global__ void dft_axis_kernel(const float2* in, float2* out, int nx, int ny, int nz, int axis, float sign)
{
    extern __shared__ float2 tw[];
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)j / (float)n, &s, &c);
        tw[j] = make_float2(c, sign * s);
    }
    __syncthreads();
    const long long N = (long long)nx * ny * nz;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 3 * N) return;
    const int comp = (int)(e / N);
    const long long r = e - comp * N;
    const int x = (int)(r % nx), y = (int)((r / nx) % ny), z = (int)(r / ((long long)nx * ny));
    const int k = axis == 0 ? x : (axis == 1 ? y : z);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : (long long)nx * ny);
    const long long base = comp * N + r - (long long)k * stride;
    float ar = 0.0f, ai = 0.0f;
    int idx = 0;
    for (int j = 0; j < n; ++j) {
        const float2 v = in[base + j * stride];
        const float2 w = tw[idx];
        ar += v.x * w.x - v.y * w.y;
        ai += v.x * w.y + v.y * w.x;
        idx += k;
        if (idx >= n) idx -= n;
    }
    out[e] = make_float2(ar, ai);
}

// u^ = P g^ / (mu |kt|^2) in place; also folds in the 1/N of the inverse DFT
__global__ void stokes_solve_kernel(float2* g, int nx, int ny, int nz, float mu)
{
    const long long N = (long long)nx * ny * nz;
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int x = (int)(r % nx), y = (int)((r / nx) % ny), z = (int)(r / ((long long)nx * ny));
    const float kx = 2.0f * sinpif((float)x / (float)nx), ky = 2.0f * sinpif((float)y / (float)ny),
                kz = 2.0f * sinpif((float)z / (float)nz);
    const float k2 = kx * kx + ky * ky + kz * kz;
    float2 a = g[r], b = g[N + r], c = g[2 * N + r];
    if (r == 0 || k2 == 0.0f) {
        a = b = c = make_float2(0.0f, 0.0f);
    } else {
        const float pr = (kx * a.x + ky * b.x + kz * c.x) / k2, pi = (kx * a.y + ky * b.y + kz * c.y) / k2;
        const float sc = 1.0f / (mu * k2 * (float)N);
        a = make_float2((a.x - kx * pr) * sc, (a.y - kx * pi) * sc);
        b = make_float2((b.x - ky * pr) * sc, (b.y - ky * pi) * sc);
        c = make_float2((c.x - kz * pr) * sc, (c.y - kz * pi) * sc);
    }
    g[r] = a;
    g[N + r] = b;
    g[2 * N + r] = c;
}

__global__ void real_part_kernel(const float2* g, long long n3, float* u)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n3) u[e] = g[e].x;
}

static unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_init_fluid(const BoxDev& B, int precision, void* fbuf, const float* u, const int* owner,
                              cudaStream_t s)
{
    const unsigned g = nblk(B.N, 256);
    if (precision == 1) init_fluid_kernel<StF16><<<g, 256, 0, s>>>(B, fbuf, u, owner);
    else if (precision == 2) init_fluid_kernel<StBF16><<<g, 256, 0, s>>>(B, fbuf, u, owner);
    else init_fluid_kernel<StF32><<<g, 256, 0, s>>>(B, fbuf, u, owner);
    return cudaGetLastError();
}

// work: 6 N float2 (two complex [3][N] buffers); counts: np + 1 ints
cudaError_t launch_stokes(const BoxDev& B, const int* owner, const PartDev* pd, int np, int counter_on,
                          const double body[3], float mu, float2* work, int* counts, float* u, cudaStream_t s)
{
    cudaError_t e;
    const long long N = B.N;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * (np + 1), s)) != cudaSuccess) return e;
    count_owner_kernel<<<nblk(N, 256), 256, 0, s>>>(owner, N, counts, np);
    float2* a = work;
    float2* b = work + 3 * N;
    force_density_kernel<<<nblk(N, 256), 256, 0, s>>>(owner, N, counts, pd, np, counter_on, body[0], body[1], body[2],
                                                       a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nmax = B.nx > B.ny ? (B.nx > B.nz ? B.nx : B.nz) : (B.ny > B.nz ? B.ny : B.nz);
    const size_t sh = sizeof(float2) * nmax;
    for (int ax = 0; ax < 3; ++ax) {
        dft_axis_kernel<<<nblk(3 * N, 256), 256, sh, s>>>(ax % 2 == 0 ? a : b, ax % 2 == 0 ? b : a, B.nx, B.ny, B.nz, ax,
                                                          -1.0f);
    }
    // forward result in b (three passes: a->b, b->a, a->b)
    stokes_solve_kernel<<<nblk(N, 256), 256, 0, s>>>(b, B.nx, B.ny, B.nz, mu);
    for (int ax = 0; ax < 3; ++ax) {
        dft_axis_kernel<<<nblk(3 * N, 256), 256, sh, s>>>(ax % 2 == 0 ? b : a, ax % 2 == 0 ? a : b, B.nx, B.ny, B.nz, ax,
                                                          1.0f);
    }
    // inverse result in a
    real_part_kernel<<<nblk(3 * N, 256), 256, 0, s>>>(a, 3 * N, u);
    return cudaGetLastError();
}

}  // namespace lbsph
