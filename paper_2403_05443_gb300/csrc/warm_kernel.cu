// Warm start of a run (lb_init_fluid, lb_stokes_field): an initial fluid at
// the local equilibrium of given velocity and density fields (optionally with
// the viscous stress of the velocity field in its non-equilibrium part), and
// the periodic steady flow (with its density) that the particles' external
// forces drive in the lattice fluid, as those fields.
//
// The force density g puts F_ext of each particle uniformly on the fluid nodes
// next to it, and the box's uniform counter force and body force on the fluid
// nodes; the mean of g (if the forces do not balance) is dropped.  The flow is
// the exact steady state of the linear lattice dynamics itself (D3Q19 BGK with
// Guo forcing, lattice_steady_kernel), not of a discretised Stokes operator:
// at the scales of a few nodes the lattice's viscous and pressure operators
// differ from any fixed stencil by several per cent, and a start that differs
// from the lattice's own steady state by that much relaxes on the flow's slow
// time scales.  The mean flow is then set so that the fluid and particle
// momenta add up to zero (rho0 sum_fluid u = -sum_p M_p U_p, with the
// particles' initial velocities), as they do in a run from rest with a
// balancing counter force.  The transforms are separable DFTs along x, y and z:
// a radix-2 FFT per line in shared memory for power-of-two edges, otherwise
// computed by definition (one output element per thread, the line's twiddle
// table in shared memory); FP32 complex, the per-mode solve in FP64.
#include "lattice_common.cuh"

namespace lbsph {

// f = f_eq(rho0 + drho, u) - w rho0 on fluid nodes (deviation storage), 0
// elsewhere; drho may be null (uniform density).  stress: plus the first-order
// non-equilibrium part -3 tau rho w_i (c_ia c_ib - delta_ab / 3) d_a u_b with
// d_a the periodic central difference (u is read on every node, solid or not)
template <class St>
__global__ void init_fluid_kernel(const BoxDev B, void* fbuf, const float* u, const float* drho, const int* owner,
                                  float tau, int stress)
{
    using T = typename St::T;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= B.N) return;
    T* f = reinterpret_cast<T*>(fbuf) + B.off;
    const bool fluid = owner[n] == 0;
    const float ux = fluid ? u[n] : 0.0f, uy = fluid ? u[B.N + n] : 0.0f, uz = fluid ? u[2 * B.N + n] : 0.0f;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float dr = (fluid && drho) ? drho[n] : 0.0f;
    const float rho = B.rho0f + dr;
    float du[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};   // du[a][b] = d_a u_b
    if (stress && fluid) {
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
        const long long row = (long long)nx * ny;
        const long long yz = (long long)z * row + (long long)y * nx;
        const long long nb[3][2] = {
            {yz + (x == nx - 1 ? 0 : x + 1), yz + (x == 0 ? nx - 1 : x - 1)},
            {(long long)z * row + (long long)(y == ny - 1 ? 0 : y + 1) * nx + x,
             (long long)z * row + (long long)(y == 0 ? ny - 1 : y - 1) * nx + x},
            {(long long)(z == nz - 1 ? 0 : z + 1) * row + (long long)y * nx + x,
             (long long)(z == 0 ? nz - 1 : z - 1) * row + (long long)y * nx + x}};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) du[a][b] = 0.5f * (u[b * B.N + nb[a][0]] - u[b * B.N + nb[a][1]]);
    }
    const float dv = (du[0][0] + du[1][1] + du[2][2]) * (1.0f / 3.0f);
    const unsigned long long pol = l2_evict_normal();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
        float d = w_of(i) * (dr + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
        if (stress) {
            const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
            float q = -dv;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    if (c[a] * c[b] != 0) q += (float)(c[a] * c[b]) * du[a][b];
            d += -3.0f * tau * rho * w_of(i) * q;
        }
        St::st1(f + (long long)i * B.N + n, fluid ? d : 0.0f, B.scale, pol);
    }
}

// shell owner of a fluid node: the particle (p + 1) owning one of its six face
// neighbours, 0 if none (periodic; the first one found if several)
__device__ __forceinline__ int shell_owner(const int* owner, int nx, int ny, int nz, long long n)
{
    const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
    const int xs[2] = {x == 0 ? nx - 1 : x - 1, x == nx - 1 ? 0 : x + 1};
    const int ys[2] = {y == 0 ? ny - 1 : y - 1, y == ny - 1 ? 0 : y + 1};
    const int zs[2] = {z == 0 ? nz - 1 : z - 1, z == nz - 1 ? 0 : z + 1};
    const long long row = (long long)nx * ny;
    int o = 0;
    for (int k = 0; k < 2; ++k) {
        const int a = owner[z * row + (long long)y * nx + xs[k]];
        const int b = owner[z * row + (long long)ys[k] * nx + x];
        const int c = owner[zs[k] * row + (long long)y * nx + x];
        if (o == 0 && a > 0) o = a;
        if (o == 0 && b > 0) o = b;
        if (o == 0 && c > 0) o = c;
    }
    return o;
}

// shell-node count of each particle of the box (fluid nodes next to it) and
// fluid count
__global__ void count_owner_kernel(const int* owner, int nx, int ny, int nz, int* counts, int np)
{
    const long long N = (long long)nx * ny * nz;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N || owner[n] != 0) return;
    atomicAdd(counts, 1);
    const int o = shell_owner(owner, nx, ny, nz, n);
    if (o > 0 && o <= np) atomicAdd(counts + o, 1);
}

// force density as complex [3][N]: F_ext / nshell on the fluid nodes next to
// a particle (a uniform traction just outside its surface, under which a
// sphere's interior moves rigidly at its Stokes velocity), plus the body force
// and (counter_on) -sum F_ext / N_fluid on every fluid node
__global__ void force_density_kernel(const int* owner, int nx, int ny, int nz, const int* counts, const PartDev* pd,
                                     int np, int counter_on, double bx, double by, double bz, float2* g)
{
    const long long N = (long long)nx * ny * nz;
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    double f[3] = {0.0, 0.0, 0.0};
    if (owner[n] == 0) {
        f[0] = bx; f[1] = by; f[2] = bz;
        if (counter_on && counts[0] > 0) {
            for (int p = 0; p < np; ++p)
                for (int k = 0; k < 3; ++k) f[k] -= pd[p].Fext[k] / (double)counts[0];
        }
        const int o = shell_owner(owner, nx, ny, nz, n);
        if (o > 0 && o <= np) {
            const double c = 1.0 / (double)counts[o];
            for (int k = 0; k < 3; ++k) f[k] += pd[o - 1].Fext[k] * c;
        }
    }
    for (int k = 0; k < 3; ++k) g[k * N + n] = make_float2((float)f[k], 0.0f);
}

// one DFT pass along one axis: out(.., k, ..) = sum_j in(.., j, ..) w^(j k),
// w = exp(sign 2 pi i / n); ncomp components of [nz][ny][nx] each
__global__ void dft_axis_kernel(const float2* in, float2* out, int nx, int ny, int nz, int axis, float sign,
                                int ncomp)
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
    if (e >= ncomp * N) return;
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

// the same pass for a power-of-two length n = 2^logn: one block per line, the
// line staged in shared memory in bit-reversed order and transformed by logn
// radix-2 butterfly stages (decimation in time) with the twiddles of the line
// in shared memory; O(n log n) instead of O(n^2) per line
__global__ void fft_axis_kernel(const float2* in, float2* out, int nx, int ny, int nz, int axis, float sign, int logn)
{
    extern __shared__ float2 fsm[];
    const int n = 1 << logn;
    float2* buf = fsm;
    float2* tw = fsm + n;
    const long long N = (long long)nx * ny * nz;
    const long long lines = N / n;                  // lines of one component
    const int comp = (int)(blockIdx.x / lines);
    const long long l = blockIdx.x - comp * lines;
    long long base, stride;
    if (axis == 0) {
        stride = 1;
        base = comp * N + l * nx;
    } else if (axis == 1) {
        stride = nx;
        base = comp * N + (l / nx) * ((long long)nx * ny) + (l % nx);
    } else {
        stride = (long long)nx * ny;
        base = comp * N + l;                        // l = y * nx + x
    }
    for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
        float sn, cs;
        sincospif(2.0f * (float)j / (float)n, &sn, &cs);
        tw[j] = make_float2(cs, sign * sn);
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int rj = (int)(__brev((unsigned)j) >> (32 - logn));
        buf[rj] = in[base + j * stride];
    }
    __syncthreads();
    for (int st = 1; st <= logn; ++st) {
        const int half = 1 << (st - 1);
        for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
            const int grp = t >> (st - 1), pos = t & (half - 1);
            const int i0 = (grp << st) + pos, i1 = i0 + half;
            const float2 w = tw[pos << (logn - st)];
            const float2 a = buf[i0], b = buf[i1];
            const float2 bw = make_float2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
            buf[i0] = make_float2(a.x + bw.x, a.y + bw.y);
            buf[i1] = make_float2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) out[base + j * stride] = buf[j];
}

static int log2_if_pow2(int n)
{
    if (n < 2 || (n & (n - 1)) != 0) return -1;
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Steady state of the linear lattice fluid itself (D3Q19 BGK, omega = 1/tau,
// Guo forcing, about rho0) under the force density g, mode by mode (k = 2 pi
// (x/nx, y/ny, z/nz) for the DFT index (x, y, z)).  The steady pre-collision
// populations are the post-collision ones streamed, f^_i = e_i f^*_i with
// e_i = exp(-i k.c_i), hence f^_i = h_i (omega f^eq_i + (1 - omega/2) F^_i),
// h_i = e_i / (1 - (1 - omega) e_i), F_i = 3 w_i c_i.g, and their moments
// (drho, u = j + g/2) solve
//   D0 drho - 3 rho0 omega H1 . u = 3 (1 - omega/2) H1 . g
//   -omega H1 drho + rho0 D2 u     = g/2 + 3 (1 - omega/2) H2 g
// with H1 = sum w_i c_i h_i, H2 = sum w_i c_i c_i^T h_i,
// D0 = sum w_i (1 - e_i) q_i and D2 = sum 3 w_i c_i c_i^T (1 - e_i) q_i,
// q_i = 1 / (1 - (1 - omega) e_i), with 1 - e_i = 2 sin^2(th/2) + i sin th
// written without cancellation (D0 and D2 vanish like k^2).  The terms of one
// direction in FP32, their sums and the solve in FP64 (Gaussian elimination
// with partial pivoting); the k = 0 mode (mean flow and
// mass, set afterwards) and numerically singular modes are zero.  On entry g
// holds the transformed force density (components 0-2); on exit u^ (0-2) and
// drho^ (3), with the 1/N of the inverse DFT folded in.
struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b)
{
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return {a.re * s, a.im * s}; }

__global__ void lattice_steady_kernel(float2* g, int nx, int ny, int nz, double omega, double rho0)
{
    const long long N = (long long)nx * ny * nz;
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int x = (int)(r % nx), y = (int)((r / nx) % ny), z = (int)(r / ((long long)nx * ny));
    cplx H1[3] = {}, H2[3][3] = {}, D0 = {}, D2[3][3] = {};
    // each direction's terms in FP32 (the terms of c and -c are exact complex
    // conjugates, so the imaginary parts still cancel pairwise), summed in FP64
    const float fx = (float)x / nx, fy = (float)y / ny, fz = (float)z / nz, om1 = (float)(1.0 - omega);
#pragma unroll
    for (int i = 1; i < Q; ++i) {        // the rest population has c = 0: no share in H1, H2, D0, D2
        const int c[3] = {cx_of(i), cy_of(i), cz_of(i)};
        // theta / pi, reduced to [-1, 1) so that sinpi / cospi stay exact at multiples of pi
        float tp = 2.0f * (fx * c[0] + fy * c[1] + fz * c[2]);
        tp -= 2.0f * floorf(0.5f * tp + 0.5f);
        float snf, csf;
        sincospif(tp, &snf, &csf);
        const float shf = sinpif(0.5f * tp);
        const float dre = 1.0f - om1 * csf, dim = om1 * snf, dd = dre * dre + dim * dim;
        // h = e / den, q = (1 - e) / den with e = cs - i sn, 1 - e = 2 sh^2 + i sn
        const float hre = (csf * dre - snf * dim) / dd, him = (-snf * dre - csf * dim) / dd;
        const float are = 2.0f * shf * shf, aim = snf;
        const float qre = (are * dre + aim * dim) / dd, qim = (aim * dre - are * dim) / dd;
        const cplx h = {(double)hre, (double)him};
        const cplx q = {(double)qre, (double)qim};
        const double w = wd_of(i);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (c[a] == 0) continue;
            H1[a] = cadd(H1[a], cscale(h, w * c[a]));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (c[b] == 0) continue;
                H2[a][b] = cadd(H2[a][b], cscale(h, w * c[a] * c[b]));
                D2[a][b] = cadd(D2[a][b], cscale(q, 3.0 * w * c[a] * c[b]));
            }
        }
        D0 = cadd(D0, cscale(q, w));
    }
    const float2 g0 = g[r], g1 = g[N + r], g2 = g[2 * N + r];
    const cplx gh[3] = {{g0.x, g0.y}, {g1.x, g1.y}, {g2.x, g2.y}};
    const double fo = 3.0 * (1.0 - 0.5 * omega);
    // augmented 4 x 5 system: unknowns (drho, ux, uy, uz)
    cplx M[4][5];
    M[0][0] = D0;
    cplx r0 = {0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        M[0][1 + a] = cscale(H1[a], -3.0 * rho0 * omega);
        r0 = cadd(r0, cmul(H1[a], gh[a]));
    }
    M[0][4] = cscale(r0, fo);
    for (int a = 0; a < 3; ++a) {
        M[1 + a][0] = cscale(H1[a], -omega);
        cplx ra = cscale(gh[a], 0.5);
        for (int b = 0; b < 3; ++b) {
            M[1 + a][1 + b] = cscale(D2[a][b], rho0);
            ra = cadd(ra, cscale(cmul(H2[a][b], gh[b]), fo));
        }
        M[1 + a][4] = ra;
    }
    double scale = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) scale = fmax(scale, fabs(M[a][b].re) + fabs(M[a][b].im));
    bool ok = r != 0 && scale > 0.0;
    for (int col = 0; col < 4 && ok; ++col) {
        int piv = col;
        double best = 0.0;
        for (int row = col; row < 4; ++row) {
            const double m = M[row][col].re * M[row][col].re + M[row][col].im * M[row][col].im;
            if (m > best) { best = m; piv = row; }
        }
        if (!(sqrt(best) > 1e-14 * scale)) { ok = false; break; }
        if (piv != col)
            for (int j = 0; j < 5; ++j) { const cplx t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
        for (int row = 0; row < 4; ++row) {
            if (row == col) continue;
            const cplx f = cdiv(M[row][col], M[col][col]);
            for (int j = col; j < 5; ++j) M[row][j] = csub(M[row][j], cmul(f, M[col][j]));
        }
    }
    cplx sol[4] = {};
    if (ok)
        for (int a = 0; a < 4; ++a) sol[a] = cscale(cdiv(M[a][4], M[a][a]), 1.0 / (double)N);
    g[r] = make_float2((float)sol[1].re, (float)sol[1].im);
    g[N + r] = make_float2((float)sol[2].re, (float)sol[2].im);
    g[2 * N + r] = make_float2((float)sol[3].re, (float)sol[3].im);
    g[3 * N + r] = make_float2((float)sol[0].re, (float)sol[0].im);
}

__global__ void real_part_kernel(const float2* g, long long n3, float* u)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n3) u[e] = g[e].x;
}

// sum over fluid nodes of u and drho (4 doubles), one atomic per warp
__global__ void fluid_sum_kernel(const float* u, const int* owner, long long N, double* sum)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (n < N && owner[n] == 0)
        for (int k = 0; k < 4; ++k) v[k] = u[k * N + n];
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if ((threadIdx.x & 31) == 0 && v[k] != 0.0) atomicAdd(sum + k, v[k]);
    }
}

// uniform shift of the fluid so that fluid + particle momentum is zero:
// rho0 sum_fluid u + sum_p M_p U_p = 0
__global__ void momentum_shift_kernel(float* u, const int* owner, long long N, const double* sum, const int* counts,
                                      const PartDev* pd, int np, double rho0)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N || owner[n] != 0 || counts[0] == 0) return;
    for (int k = 0; k < 3; ++k) {
        double P = 0.0;
        for (int p = 0; p < np; ++p) P += pd[p].M * pd[p].U[k];
        const double shift = (-P / rho0 - sum[k]) / (double)counts[0];
        u[k * N + n] += (float)shift;
    }
    u[3 * N + n] -= (float)(sum[3] / (double)counts[0]);     // no net mass change
}

static unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_init_fluid(const BoxDev& B, int precision, void* fbuf, const float* u, const float* drho,
                              const int* owner, float tau, int stress, cudaStream_t s)
{
    const unsigned g = nblk(B.N, 256);
    if (precision == 1) init_fluid_kernel<StF16><<<g, 256, 0, s>>>(B, fbuf, u, drho, owner, tau, stress);
    else if (precision == 2) init_fluid_kernel<StBF16><<<g, 256, 0, s>>>(B, fbuf, u, drho, owner, tau, stress);
    else init_fluid_kernel<StF32><<<g, 256, 0, s>>>(B, fbuf, u, drho, owner, tau, stress);
    return cudaGetLastError();
}

// work: 8 N float2 (two complex [4][N] buffers); counts: np + 1 ints; sum: 4
// doubles; u: [4][N] (velocity, then the density deviation)
cudaError_t launch_stokes(const BoxDev& B, const int* owner, const PartDev* pd, int np, int counter_on,
                          const double body[3], float2* work, int* counts, double* sum, float* u,
                          cudaStream_t s)
{
    cudaError_t e;
    const long long N = B.N;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(int) * (np + 1), s)) != cudaSuccess) return e;
    count_owner_kernel<<<nblk(N, 256), 256, 0, s>>>(owner, B.nx, B.ny, B.nz, counts, np);
    float2* a = work;
    float2* b = work + 4 * N;
    force_density_kernel<<<nblk(N, 256), 256, 0, s>>>(owner, B.nx, B.ny, B.nz, counts, pd, np, counter_on, body[0],
                                                       body[1], body[2], a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nmax = B.nx > B.ny ? (B.nx > B.nz ? B.nx : B.nz) : (B.ny > B.nz ? B.ny : B.nz);
    const size_t sh = sizeof(float2) * nmax;
    // one pass along an axis: the radix-2 FFT for power-of-two edges, else the
    // transform by definition
    auto pass = [&](const float2* src, float2* dst, int ax, float sign, int ncomp) {
        const int n = ax == 0 ? B.nx : (ax == 1 ? B.ny : B.nz);
        const int lg = log2_if_pow2(n);
        if (lg > 0) {
            const int threads = n / 2 < 32 ? 32 : (n / 2 > 256 ? 256 : n / 2);
            fft_axis_kernel<<<(unsigned)(ncomp * (N / n)), threads, sizeof(float2) * (n + n / 2), s>>>(
                src, dst, B.nx, B.ny, B.nz, ax, sign, lg);
        } else {
            dft_axis_kernel<<<nblk(ncomp * N, 256), 256, sh, s>>>(src, dst, B.nx, B.ny, B.nz, ax, sign, ncomp);
        }
    };
    for (int ax = 0; ax < 3; ++ax) pass(ax % 2 == 0 ? a : b, ax % 2 == 0 ? b : a, ax, -1.0f, 3);
    // forward result in b (three passes: a->b, b->a, a->b)
    lattice_steady_kernel<<<nblk(N, 128), 128, 0, s>>>(b, B.nx, B.ny, B.nz, (double)B.omega, B.rho0);
    for (int ax = 0; ax < 3; ++ax) pass(ax % 2 == 0 ? b : a, ax % 2 == 0 ? a : b, ax, 1.0f, 4);
    // inverse result in a
    real_part_kernel<<<nblk(4 * N, 256), 256, 0, s>>>(a, 4 * N, u);
    if ((e = cudaMemsetAsync(sum, 0, 4 * sizeof(double), s)) != cudaSuccess) return e;
    fluid_sum_kernel<<<nblk(N, 256), 256, 0, s>>>(u, owner, N, sum);
    momentum_shift_kernel<<<nblk(N, 256), 256, 0, s>>>(u, owner, N, sum, counts, pd, np, B.rho0);
    return cudaGetLastError();
}

}  // namespace lbsph
