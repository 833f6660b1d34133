// Host runtime behind the C ABI of include/lbsph.h.
//
// One iteration has four parts: the bulk lattice part (every node but those
// next to a particle's surface), the boundary part (the nodes the bulk part
// skips, written into the same lattice buffer), the critical particle part
// (solve, pose, new occupancy, redo masks and box forces for the next step)
// and the auxiliary particle part (drag matrices and the inverse of the next
// solve).  Time steps run in the persistent step kernel (step_kernel.cu), many
// iterations per cooperative launch; the first collision, the per-kernel
// profile and LB_FLAG_SEPARATE_KERNELS run the four parts as separate kernels
// in stream order.  Everything runs on the caller's stream.  Chunks of iterations are captured
// once into a CUDA graph per buffer parity and replayed, so a long run costs
// one graph launch per chunk and no host synchronisation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbsph.h"
#include "lbsph_internal.cuh"
#include "q27.cuh"

namespace lbsph {
cudaError_t launch_fields(const KParams& p, int precision, int blocks, cudaStream_t s);
cudaError_t launch_bulk(const BulkParams& p, int precision, int blocks, cudaStream_t s);
cudaError_t launch_boundary(const BndParams& p, int precision, int np, cudaStream_t s);
cudaError_t launch_particles(const PParams& p, cudaStream_t s);
cudaError_t launch_particles_aux(const PParams& p, cudaStream_t s);
cudaError_t launch_step(const BulkParams bulk[2], const BndParams bnd[2], const PParams part[2], unsigned* sync,
                        unsigned* status, int np, int gx, int tiles, int iters, int cur0, int precision, int fetch,
                        const double* io_ft, double* io_rec, cudaStream_t s);
cudaError_t launch_links(const PartDev* pd, const PartK* pk, const uint64_t* rows, const BoxDev* boxes, int p, int* out,
                         int cap, int* count, cudaStream_t s);
cudaError_t launch_init_fluid(const BoxDev& B, int precision, void* fbuf, const float* u, const float* drho,
                              const int* owner, float tau, int stress, cudaStream_t s);
cudaError_t launch_stokes(const BoxDev& B, const int* owner, const PartDev* pd, int np, int counter_on,
                          const double body[3], float2* work, int* counts, double* sum, float* u,
                          cudaStream_t s);
}  // namespace lbsph

using namespace lbsph;

namespace {
constexpr int STEP_ITERS = 256;     // iterations per launch of the step kernel
}

struct lb_ctx {
    int device = 0;
    lb_options opt{};
    cudaStream_t stream = nullptr;
    std::vector<lb_box_desc> desc;
    std::vector<BoxDev> hbox;
    BoxDev* d_boxes = nullptr;
    int total_blocks = 0;
    size_t elem = 4;
    long long total_elems = 0;
    void* fbuf[2] = {nullptr, nullptr};
    int cur = 0;                        // fbuf[cur] holds the latest populations
    int maxp = 0;
    int np = 0;
    std::vector<std::vector<lb_particle>> parts;
    PartDev* d_pd = nullptr;
    PartK* d_pk = nullptr;
    long long* d_acc = nullptr;
    uint64_t* d_rows = nullptr;
    unsigned* d_status = nullptr;
    int* d_links = nullptr;
    int links_cap = 0;
    int* d_count = nullptr;
    float* d_tmp = nullptr;
    float2* d_stokes = nullptr;         // lb_stokes_field: two complex [3][N] buffers of the largest box
    int* d_counts = nullptr;
    double* d_rec = nullptr;
    size_t tmp_bytes = 0;
    bool collided = false;
    bool stepped = false;
    unsigned sticky = 0;
    cudaStream_t last_user_stream = nullptr;        // last stream lb_step ran on
    cudaEvent_t ev_done = nullptr;                  // end of the last lb_step
    unsigned* d_sync = nullptr;                     // step kernel: barrier, work and item counters, block SM ids
    double* d_ring = nullptr;                       // [maxp][2][RINGD] poses of the last two times (partners)
    NeedHdr* d_need_hdr = nullptr;     // [2][maxp]: redo masks, one slot per buffer parity
    uint64_t* d_need = nullptr;        // [2][maxp][MAXS*MAXS]
    int* d_blk_box = nullptr;
    BoxDyn* d_box_dyn = nullptr;       // [2][nbox]: one slot per buffer parity
    BoxDyn* d_pdyn = nullptr;          // [2][maxp]: the same per particle
    int* d_box_done = nullptr;
    int list_cap = 0;                  // node list entries per boundary block
    int gx = 1;                        // boundary blocks per particle
    int fetch = 1;                     // bulk units a warp takes per counter fetch (lb_autotune)
    int kprec = 0;                     // kernel variant: precision, or 3 for FP32 with the ghost-mode collision
    bool aux_pending = false;          // the auxiliary particle blocks of the last step kernel's
                                       // last iteration have not run yet (the next launch runs them)
    std::string err;
    std::vector<void*> allocs;
    // D3Q27 (lb_options.lattice = 27): q27.cuh
    int lattice = 19;
    std::vector<q27::Box27> h27;
    std::vector<q27::Part27> hpart27;  // host copies of the particles as set
    std::vector<int> box27_part;       // particle slot of every box, or -1
    q27::Box27* d_box27 = nullptr;
    q27::Dyn27* d_dyn27 = nullptr;
    q27::Part27* d_part27 = nullptr;
    int* d_blk27 = nullptr;
    int blocks27 = 0;
    int dpar27 = 0;                    // slot of d_dyn27 ([2][nbox]) the next lattice pass reads
    int nbpp27 = 1;                    // near-pass blocks per particle
    cudaStream_t s27 = nullptr;        // near pass and particle kernel, beside the bulk pass
    cudaEvent_t ev27a = nullptr, ev27b = nullptr;
};

static lb_status fail(lb_ctx* c, lb_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

static lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, LB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

static void* dev_alloc(lb_ctx* ctx, size_t bytes)
{
    void* p = nullptr;
    if (bytes == 0) bytes = 256;
    if (ctx->opt.alloc) {
        p = ctx->opt.alloc(bytes, ctx->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->allocs.push_back(p);
    return p;
}

static void free_all(lb_ctx* ctx)
{
    for (void* p : ctx->allocs) {
        if (ctx->opt.alloc && ctx->opt.release) ctx->opt.release(p, ctx->opt.alloc_user);
        else if (!ctx->opt.alloc) cudaFree(p);
    }
    ctx->allocs.clear();
}

static cudaStream_t pick(lb_ctx* ctx, void* s) { return s ? static_cast<cudaStream_t>(s) : ctx->stream; }

// errors are returned by the call that caused them; drop a stale one so that a
// later cudaGetLastError() after a launch reports that launch only
static void clear_stale_error() { (void)cudaGetLastError(); }

static lb_status read_status(lb_ctx* ctx)
{
    unsigned st = 0;
    CK(cudaMemcpy(&st, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    ctx->sticky |= st;
    if (ctx->sticky & ST_NAN) return fail(ctx, LB_ENAN, "a particle state became NaN or Inf");
    if (ctx->sticky & ST_OVERLAP) return fail(ctx, LB_EOVERLAP, "a particle reached a wall or another particle");
    if (ctx->sticky & ST_CAPACITY) return fail(ctx, LB_ECAPACITY, "a particle outgrew its bounding cube or a tile met too many particles");
    if (ctx->sticky & ST_TIMEOUT) return fail(ctx, LB_ECUDA, "a grid barrier of the step kernel timed out");
    return LB_OK;
}

// ---------------------------------------------------------------------------
extern "C" int32_t lb_abi_version(void) { return LBSPH_ABI_VERSION; }

extern "C" const char* lb_status_string(lb_status s)
{
    switch (s) {
    case LB_OK: return "ok";
    case LB_EINVAL: return "invalid argument";
    case LB_ENOMEM: return "out of device memory";
    case LB_ECUDA: return "CUDA error";
    case LB_ETIMEOUT: return "device wait timed out";
    case LB_ENAN: return "particle state is not finite";
    case LB_EOVERLAP: return "particles overlap";
    case LB_ECAPACITY: return "capacity exceeded";
    case LB_ESTATE: return "call not allowed in this state";
    }
    return "unknown status";
}

extern "C" const char* lb_last_error(const lb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" void lb_lattice(int32_t* c57, double* w19)
{
    for (int i = 0; i < Q; ++i) {
        if (c57) { c57[3 * i] = cx_of(i); c57[3 * i + 1] = cy_of(i); c57[3 * i + 2] = cz_of(i); }
        if (w19) w19[i] = wd_of(i);
    }
}

extern "C" lb_status lb_lattice_q(int32_t q, int32_t* c, double* w)
{
    if (q != 19 && q != 27) return LB_EINVAL;
    for (int i = 0; i < q; ++i) {
        if (c) { c[3 * i] = q27::cx27(i); c[3 * i + 1] = q27::cy27(i); c[3 * i + 2] = q27::cz27(i); }
        if (w) w[i] = q == 19 ? wd_of(i) : q27::wd27(i);
    }
    return LB_OK;
}

// ---------------------------------------------------------------------------
// D3Q27 path (q27.cuh): the context's boxes, at most one passive particle per
// box, two kernels per iteration.
static lb_status q27_create(lb_ctx* ctx, const lb_box_desc* boxes, int nbox)
{
    const lb_options& o = ctx->opt;
    if (o.precision != LB_FP32) return fail(ctx, LB_EINVAL, "D3Q27: FP32 storage only");
    for (int b = 0; b < nbox; ++b)
        if (boxes[b].walls) return fail(ctx, LB_EINVAL, "D3Q27: periodic boxes only");
    ctx->lattice = 27;
    ctx->elem = 4;
    ctx->maxp = nbox;
    ctx->desc.assign(boxes, boxes + nbox);
    ctx->parts.assign(nbox, {});
    ctx->box27_part.assign(nbox, -1);
    long long off = 0;
    int blk = 0;
    std::vector<int> blk_box;
    size_t tmp = 0;
    for (int b = 0; b < nbox; ++b) {
        const lb_box_desc& d = boxes[b];
        q27::Box27 h{};
        h.nx = d.nx; h.ny = d.ny; h.nz = d.nz; h.counter = d.counter_force;
        h.N = (long long)d.nx * d.ny * d.nz;
        h.off = off;
        off += 27 * h.N;
        h.block_begin = blk;
        h.nblocks = (int)((h.N + 255) / 256);
        for (int k = 0; k < h.nblocks; ++k) blk_box.push_back(b);
        blk += h.nblocks;
        h.omega = (float)(1.0 / d.tau);
        h.rho0 = d.rho0;
        h.rho0f = (float)d.rho0;
        for (int k = 0; k < 3; ++k) h.body[k] = d.body_force[k];
        h.p = -1;
        magic_div((unsigned)d.nx, h.dx_m, h.dx_s);
        magic_div((unsigned)d.ny, h.dy_m, h.dy_s);
        if (27ll * h.N >= (1ll << 31)) return fail(ctx, LB_EINVAL, "D3Q27: box too large (27 N >= 2^31)");
        ctx->h27.push_back(h);
        tmp = std::max(tmp, (size_t)(27 * h.N) * sizeof(float));
    }
    ctx->blocks27 = blk;
    ctx->total_elems = off;
    ctx->tmp_bytes = tmp;
    ctx->fbuf[0] = dev_alloc(ctx, (size_t)off * 4);
    ctx->fbuf[1] = dev_alloc(ctx, (size_t)off * 4);
    ctx->d_box27 = (q27::Box27*)dev_alloc(ctx, sizeof(q27::Box27) * nbox);
    ctx->d_dyn27 = (q27::Dyn27*)dev_alloc(ctx, sizeof(q27::Dyn27) * 2 * nbox);
    ctx->d_part27 = (q27::Part27*)dev_alloc(ctx, sizeof(q27::Part27) * nbox);
    ctx->d_blk27 = (int*)dev_alloc(ctx, sizeof(int) * (size_t)blk);
    ctx->d_rows = (uint64_t*)dev_alloc(ctx, sizeof(uint64_t) * 2ull * MAXS * MAXS * nbox);
    ctx->d_acc = (long long*)dev_alloc(ctx, sizeof(long long) * NACC * nbox);
    ctx->d_status = (unsigned*)dev_alloc(ctx, sizeof(unsigned) * 4);
    ctx->d_count = (int*)dev_alloc(ctx, sizeof(int) * 4);
    for (void* q : {ctx->fbuf[0], ctx->fbuf[1], (void*)ctx->d_box27, (void*)ctx->d_dyn27, (void*)ctx->d_part27,
                    (void*)ctx->d_blk27, (void*)ctx->d_rows, (void*)ctx->d_acc, (void*)ctx->d_status,
                    (void*)ctx->d_count})
        if (!q) return fail(ctx, LB_ENOMEM, "D3Q27 state");
    // fluid at rest: every deviation 0
    CK(cudaMemsetAsync(ctx->fbuf[0], 0, (size_t)off * 4, ctx->stream));
    CK(cudaMemsetAsync(ctx->fbuf[1], 0, (size_t)off * 4, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_acc, 0, sizeof(long long) * NACC * nbox, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned) * 4, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_blk27, blk_box.data(), sizeof(int) * blk_box.size(), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<q27::Dyn27> dyn(nbox);
    for (int b = 0; b < nbox; ++b) {
        dyn[b] = q27::Dyn27{};
        for (int k = 0; k < 3; ++k) dyn[b].g[k] = (float)boxes[b].body_force[k];
    }
    for (int slot = 0; slot < 2; ++slot)
        CK(cudaMemcpyAsync(ctx->d_dyn27 + slot * nbox, dyn.data(), sizeof(q27::Dyn27) * nbox, cudaMemcpyHostToDevice,
                           ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_box27, ctx->h27.data(), sizeof(q27::Box27) * nbox, cudaMemcpyHostToDevice, ctx->stream));
    // the near pass and the particle kernel are the step's critical chain: the
    // highest stream priority places their blocks before waiting bulk blocks
    int prio_lo = 0, prio_hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    CK(cudaStreamCreateWithPriority(&ctx->s27, cudaStreamNonBlocking, prio_hi));
    CK(cudaEventCreateWithFlags(&ctx->ev27a, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev27b, cudaEventDisableTiming));
    CK(cudaStreamSynchronize(ctx->stream));
    return LB_OK;
}

static lb_status q27_set_particles(lb_ctx* ctx, int box, const lb_particle* p, int n)
{
    if (n > 1) return fail(ctx, LB_EINVAL, "D3Q27: at most one particle per box");
    const lb_box_desc& d = ctx->desc[box];
    if (n == 1) {
        const lb_particle& P = p[0];
        const double m = std::max(P.semi[0], std::max(P.semi[1], P.semi[2]));
        const double qn2 = P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3];
        if (!(P.semi[0] > 0 && P.semi[1] > 0 && P.semi[2] > 0) || !(m <= ctx->opt.max_semi) || !(P.density > 0) ||
            !(qn2 > 0) || !std::isfinite(qn2))
            return fail(ctx, LB_EINVAL, "bad particle");
        if (P.B1 != 0.0 || P.B2 != 0.0) return fail(ctx, LB_EINVAL, "D3Q27: passive particles only (B1 = B2 = 0)");
        const int h = (int)std::ceil(m) + CUBE_MARGIN, S = 2 * h + 2;
        if (d.nx < S + 2 || d.ny < S + 2 || d.nz < S + 2)
            return fail(ctx, LB_EINVAL, "box smaller than the particle's bounding cube");
    }
    ctx->parts[box].assign(p, p + n);
    // particle slots in box order
    ctx->hpart27.clear();
    int np = 0;
    for (int b = 0; b < (int)ctx->desc.size(); ++b) {
        ctx->box27_part[b] = ctx->parts[b].empty() ? -1 : np++;
        ctx->h27[b].p = ctx->box27_part[b];
        if (ctx->parts[b].empty()) continue;
        const lb_particle& P = ctx->parts[b][0];
        q27::Part27 D{};
        const double a = P.semi[0], bb = P.semi[1], c = P.semi[2];
        for (int k = 0; k < 3; ++k) {
            D.semi[k] = P.semi[k];
            D.Fext[k] = P.F_ext[k];
            D.Text[k] = P.T_ext[k];
            D.x[k] = P.x[k];
            D.U[k] = P.U[k];
            D.W[k] = P.Omega[k];
        }
        // Eq. vectrotn needs |q| = 1: divided by sqrt of the squares summed in order
        const double qn = std::sqrt(P.q[0] * P.q[0] + P.q[1] * P.q[1] + P.q[2] * P.q[2] + P.q[3] * P.q[3]);
        for (int k = 0; k < 4; ++k) D.q[k] = P.q[k] / qn;
        D.M = P.density * 4.0 / 3.0 * M_PI * a * bb * c;       // continuum volume
        D.Ib[0] = D.M * (bb * bb + c * c) / 5.0;               // Sec. II.D
        D.Ib[1] = D.M * (a * a + c * c) / 5.0;
        D.Ib[2] = D.M * (a * a + bb * bb) / 5.0;
        for (int k = 0; k < 3; ++k) D.inv2[k] = 1.0 / (P.semi[k] * P.semi[k]);   // IEEE: as the device rounds it
        // FP32 decides a node of the map when its inside value is farther than
        // this from 1: the FP32 rounding of the row quadratic near the surface
        // grows with the squared aspect ratio (the terms that cancel) and with
        // 1 / the short semi-axis (the gradient times the coordinate's rounding)
        {
            const double amax = std::max(a, std::max(bb, c)), amin = std::min(a, std::min(bb, c));
            D.band = (float)(1e-4 * (1.0 + 0.25 * (amax / amin) * (amax / amin) + 1.0 / amin));
        }
        D.h = (int)std::ceil(std::max(a, std::max(bb, c))) + CUBE_MARGIN;
        D.S = 2 * D.h + 2;
        D.box = b;
        ctx->hpart27.push_back(D);
    }
    ctx->np = np;
    cudaStream_t s = ctx->stream;
    const int nbox = (int)ctx->desc.size();
    std::vector<q27::Dyn27> dyn(nbox);
    for (int b = 0; b < nbox; ++b) {
        dyn[b] = q27::Dyn27{};
        for (int k = 0; k < 3; ++k) dyn[b].g[k] = (float)ctx->desc[b].body_force[k];
    }
    for (int slot = 0; slot < 2; ++slot)
        CK(cudaMemcpyAsync(ctx->d_dyn27 + slot * nbox, dyn.data(), sizeof(q27::Dyn27) * nbox, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_box27, ctx->h27.data(), sizeof(q27::Box27) * nbox, cudaMemcpyHostToDevice, s));
    // the near pass covers the union of a particle's old and new cubes, at most
    // (S + 1)^3 nodes while it moves less than one node per step
    long long umax = 1;
    for (const auto& D : ctx->hpart27) umax = std::max(umax, (long long)(D.S + 1) * (D.S + 1) * (D.S + 1));
    ctx->nbpp27 = (int)((umax + 255) / 256);
    if (np > 0)
        CK(cudaMemcpyAsync(ctx->d_part27, ctx->hpart27.data(), sizeof(q27::Part27) * np, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_acc, 0, sizeof(long long) * NACC * ctx->maxp, s));
    q27::PartParams27 pp{ctx->d_part27, ctx->d_dyn27 + (size_t)ctx->dpar27 * nbox, ctx->d_box27, ctx->d_rows,
                         ctx->d_acc, ctx->d_status, 1, ctx->opt.didt_mode};
    CK(q27::launch_particles27(pp, np, s));
    CK(cudaStreamSynchronize(s));
    return read_status(ctx);
}

// One step: the first collision, or a context without particles, is one
// lattice pass over every node and then the particle kernel; afterwards the
// nodes of the particles' cube unions (near pass) and the particle kernel run
// on a stream of their own beside the bulk pass over every other node, and the
// next step waits for both.  The particle kernel writes the box terms of the
// next pass into the other slot of d_dyn27, so the bulk pass never reads a slot
// that is being written.
static cudaError_t q27_enqueue(lb_ctx* ctx, int nsteps, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const size_t nbox = ctx->desc.size();
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        const q27::Dyn27* dcur = ctx->d_dyn27 + (size_t)ctx->dpar27 * nbox;
        q27::Dyn27* dnext = ctx->d_dyn27 + (size_t)(ctx->dpar27 ^ 1) * nbox;
        q27::LatParams27 lp{ctx->d_box27, dcur, ctx->d_part27, ctx->d_blk27, ctx->d_rows, ctx->d_acc,
                            (const float*)ctx->fbuf[ctx->cur], (float*)ctx->fbuf[ctx->cur ^ 1], ctx->collided ? 0 : 1,
                            q27::LAT_ALL, ctx->nbpp27, ctx->opt.collision};
        q27::PartParams27 pp{ctx->d_part27, dnext, ctx->d_box27, ctx->d_rows, ctx->d_acc, ctx->d_status, 0,
                             ctx->opt.didt_mode};
        if (ctx->collided && ctx->np == 0) {
            // no particle in any box: every node takes the plain pull and the collision
            q27::LatParams27 bulk = lp;
            bulk.mode = q27::LAT_BULK;
            if ((e = q27::launch_bulk27(bulk, ctx->blocks27, s)) != cudaSuccess) break;
        } else if (!ctx->collided) {
            if ((e = q27::launch_lattice27(lp, ctx->blocks27, s)) != cudaSuccess) break;
            if ((e = q27::launch_particles27(pp, ctx->np, s)) != cudaSuccess) break;
        } else {
            if ((e = cudaEventRecord(ctx->ev27a, s)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(ctx->s27, ctx->ev27a, 0)) != cudaSuccess) break;
            q27::LatParams27 near = lp;
            near.mode = q27::LAT_NEAR;
            if ((e = q27::launch_lattice27(near, ctx->np * ctx->nbpp27, ctx->s27)) != cudaSuccess) break;
            if ((e = q27::launch_particles27(pp, ctx->np, ctx->s27)) != cudaSuccess) break;
            q27::LatParams27 bulk = lp;
            bulk.mode = q27::LAT_BULK;
            if ((e = q27::launch_bulk27(bulk, ctx->blocks27, s)) != cudaSuccess) break;
            if ((e = cudaEventRecord(ctx->ev27b, ctx->s27)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(s, ctx->ev27b, 0)) != cudaSuccess) break;
        }
        ctx->cur ^= 1;
        ctx->dpar27 ^= 1;
        ctx->collided = true;
    }
    return e;
}

static lb_status q27_get_fields(lb_ctx* ctx, int box, uint32_t what, void* dst, size_t dst_bytes, int dst_is_device,
                                cudaStream_t s)
{
    const q27::Box27& B = ctx->h27[box];
    size_t need = 0;
    switch (what) {
    case LB_FIELD_F: case LB_FIELD_DF: need = 27ull * B.N * 4; break;
    case LB_FIELD_RHO: case LB_FIELD_SOLID: need = (size_t)B.N * 4; break;
    case LB_FIELD_U: need = 3ull * B.N * 4; break;
    default: return fail(ctx, LB_EINVAL, "exactly one LB_FIELD_* bit");
    }
    if (dst_bytes != need) return fail(ctx, LB_EINVAL, "dst_bytes does not match the field size");
    if (!ctx->d_tmp) {
        ctx->d_tmp = (float*)dev_alloc(ctx, ctx->tmp_bytes);
        if (!ctx->d_tmp) return fail(ctx, LB_ENOMEM, "field staging buffer");
    }
    q27::FieldParams27 fp{};
    fp.boxes = ctx->d_box27; fp.dyn = ctx->d_dyn27 + (size_t)ctx->dpar27 * ctx->desc.size(); fp.rows = ctx->d_rows;
    fp.src = (const float*)ctx->fbuf[ctx->cur];
    fp.box = box;
    fp.nopull = ctx->collided ? 0 : 1;
    fp.out_dev = what == LB_FIELD_DF ? 1 : 0;
    if (what == LB_FIELD_F || what == LB_FIELD_DF) fp.out_f = ctx->d_tmp;
    if (what == LB_FIELD_RHO) fp.out_rho = ctx->d_tmp;
    if (what == LB_FIELD_U) fp.out_u = ctx->d_tmp;
    if (what == LB_FIELD_SOLID) fp.out_solid = (int*)ctx->d_tmp;
    CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    CK(q27::launch_fields27(fp, B.nblocks, s));
    CK(cudaMemcpyAsync(dst, ctx->d_tmp, need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return read_status(ctx);
}

extern "C" lb_status lb_create(const lb_box_desc* boxes, int32_t nbox, const lb_options* opt, lb_ctx** out)
{
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (!boxes || nbox <= 0) return LB_EINVAL;
    lb_ctx* ctx = new (std::nothrow) lb_ctx();
    if (!ctx) return LB_ENOMEM;
    if (opt) ctx->opt = *opt;
    else {
        ctx->opt.max_semi = 16;
        ctx->opt.max_particles = 64;
    }
    lb_options& o = ctx->opt;
    if (o.max_semi <= 0) o.max_semi = 16;
    if (o.max_particles <= 0) o.max_particles = 64;
    auto bad = [&](const std::string& m) { delete ctx; (void)m; return LB_EINVAL; };
    if (o.precision < 0 || o.precision > 2 || o.didt_mode < 0 || o.didt_mode > 2 || o.max_semi > 29 ||
        o.collision < 0 || o.collision > 1 || (o.collision == 1 && o.precision != LB_FP32) ||
        (o.lattice != 0 && o.lattice != 19 && o.lattice != 27) ||
        (o.lattice == 27 && o.precision != LB_FP32) ||
        (o.alloc && !o.release) || (!o.alloc && o.release))
        return bad("options");
    for (int b = 0; b < nbox; ++b) {
        const lb_box_desc& d = boxes[b];
        // rows are moved in 16-byte units: nx a multiple of 4 (8 for 16-bit storage)
        if (d.nx < 4 || d.ny < 4 || d.nz < 4 || d.nx % (o.precision == LB_FP32 ? 4 : 8) != 0) return bad("box size");
        if (!(d.tau > 0.5) || !(d.rho0 > 0.0) || (d.walls && d.ny < 5) || !(d.lub_cut >= 0.0) || d.lub_cut > 4.0 ||
            (o.lattice == 27 && d.walls))
            return bad("box parameters");
        if ((long long)d.nx * d.ny * d.nz > (1ll << 31) / 19) return bad("box too large");
    }
    ctx->device = o.device;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) { delete ctx; return LB_ECUDA; }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming) != cudaSuccess) {
        delete ctx;
        return LB_ECUDA;
    }
    if (o.lattice == 27) {
        const lb_status r = q27_create(ctx, boxes, nbox);
        if (r != LB_OK) {
            cudaStreamSynchronize(ctx->stream);
            free_all(ctx);
            if (ctx->s27) cudaStreamDestroy(ctx->s27);
            if (ctx->ev27a) cudaEventDestroy(ctx->ev27a);
            if (ctx->ev27b) cudaEventDestroy(ctx->ev27b);
            cudaStreamDestroy(ctx->stream);
            cudaEventDestroy(ctx->ev_done);
            delete ctx;
            return r;
        }
        *out = ctx;
        return LB_OK;
    }
    ctx->elem = o.precision == LB_FP32 ? 4 : 2;
    ctx->kprec = o.collision == 1 ? 3 : o.precision;
    const float scale = o.precision == LB_FP16 ? (float)(o.fp16_scale > 0 ? o.fp16_scale : 16384.0) : 1.0f;
    ctx->desc.assign(boxes, boxes + nbox);
    ctx->parts.assign(nbox, {});
    long long off = 0;
    int blk = 0;
    for (int b = 0; b < nbox; ++b) {
        const lb_box_desc& d = boxes[b];
        BoxDev h{};
        h.nx = d.nx; h.ny = d.ny; h.nz = d.nz; h.nxq = d.nx / 4;
        h.N = (long long)d.nx * d.ny * d.nz;
        h.nq = h.N / 4;
        h.off = off;
        off += 19 * h.N;
        h.block_begin = blk;
        h.nblocks = (int)((h.nq + KBLOCK - 1) / KBLOCK);
        blk += h.nblocks;
        h.omega = (float)(1.0 / d.tau);
        h.rho0 = d.rho0;
        h.rho0f = (float)d.rho0;
        for (int k = 0; k < 3; ++k) {
            h.body[k] = d.body_force[k];
            h.uw_lo[k] = (float)d.wall_u_lo[k];
            h.uw_hi[k] = (float)d.wall_u_hi[k];
        }
        h.counter = d.counter_force;
        h.walls = d.walls;
        h.lub_cut = d.lub_cut;
        h.mu = d.rho0 * (d.tau - 0.5) / 3.0;
        h.nwall = d.walls ? 2ll * d.nx * d.nz : 0;
        h.scale = scale;
        h.inv_scale = 1.0f / scale;
        magic_div((unsigned)h.nxq, h.dq_m, h.dq_s);
        magic_div((unsigned)h.ny, h.dy_m, h.dy_s);
        h.rowwarp = (32 % h.nxq) == 0;
        ctx->hbox.push_back(h);
    }
    ctx->total_blocks = blk;
    ctx->total_elems = off;
    ctx->maxp = o.max_particles;
    size_t tmp = 0;
    for (auto& h : ctx->hbox) tmp = std::max(tmp, (size_t)(19 * h.N) * sizeof(float));
    ctx->tmp_bytes = tmp;
    bool okm = true;
    ctx->fbuf[0] = dev_alloc(ctx, (size_t)off * ctx->elem);
    ctx->fbuf[1] = dev_alloc(ctx, (size_t)off * ctx->elem);
    ctx->d_boxes = (BoxDev*)dev_alloc(ctx, sizeof(BoxDev) * nbox);
    ctx->d_pd = (PartDev*)dev_alloc(ctx, sizeof(PartDev) * ctx->maxp);
    ctx->d_pk = (PartK*)dev_alloc(ctx, sizeof(PartK) * ctx->maxp);
    ctx->d_acc = (long long*)dev_alloc(ctx, sizeof(long long) * NACC * ctx->maxp);
    ctx->d_rows = (uint64_t*)dev_alloc(ctx, sizeof(uint64_t) * 2ull * MAXS * MAXS * ctx->maxp);
    ctx->d_status = (unsigned*)dev_alloc(ctx, sizeof(unsigned) * 4);
    ctx->d_count = (int*)dev_alloc(ctx, sizeof(int) * 4);
    ctx->d_blk_box = (int*)dev_alloc(ctx, sizeof(int) * (size_t)blk);
    ctx->d_box_dyn = (BoxDyn*)dev_alloc(ctx, sizeof(BoxDyn) * 2 * nbox);   // one slot per buffer parity
    ctx->d_pdyn = (BoxDyn*)dev_alloc(ctx, sizeof(BoxDyn) * 2 * ctx->maxp);
    ctx->d_box_done = (int*)dev_alloc(ctx, sizeof(int) * nbox);
    {
        // block c of a particle takes the cube rows c, c + gx, ... (at most
        // BBLOCK of them); the boundary nodes of a spheroid filling its cube
        // number about 2-3 Smax^2, split evenly over the gx blocks
        const long long Smax = 2ll * (o.max_semi + CUBE_MARGIN) + 2;
        ctx->gx = (int)std::max(1ll, (3 * Smax * Smax + BBLOCK - 1) / BBLOCK);
        const long long total = std::min(Smax * Smax * Smax, 16 * Smax * Smax);
        ctx->list_cap = (int)((total + ctx->gx - 1) / ctx->gx);
    }
    ctx->d_need_hdr = (NeedHdr*)dev_alloc(ctx, sizeof(NeedHdr) * 2 * (size_t)ctx->maxp);
    ctx->d_need = (uint64_t*)dev_alloc(ctx, sizeof(uint64_t) * 2 * (size_t)MAXS * MAXS * ctx->maxp);
    ctx->d_sync = (unsigned*)dev_alloc(ctx, sizeof(unsigned) * (SYNC_HDR + (size_t)ctx->maxp + 2 * 4096));
    ctx->d_ring = (double*)dev_alloc(ctx, sizeof(double) * 2 * RINGD * (size_t)ctx->maxp);
    for (void* p : {ctx->fbuf[0], ctx->fbuf[1], (void*)ctx->d_boxes, (void*)ctx->d_pd, (void*)ctx->d_pk,
                    (void*)ctx->d_acc, (void*)ctx->d_rows, (void*)ctx->d_status, (void*)ctx->d_count,
                    (void*)ctx->d_blk_box, (void*)ctx->d_box_dyn, (void*)ctx->d_pdyn, (void*)ctx->d_box_done,
                    (void*)ctx->d_need_hdr, (void*)ctx->d_need, (void*)ctx->d_sync, (void*)ctx->d_ring})
        okm = okm && p;
    if (!okm) {
        free_all(ctx);
        cudaStreamDestroy(ctx->stream);
        cudaEventDestroy(ctx->ev_done);
        delete ctx;
        return LB_ENOMEM;
    }
    std::vector<int> blk_box(blk);
    std::vector<BoxDyn> dyn(2 * nbox);
    for (int b = 0; b < nbox; ++b) {
        for (int k = 0; k < ctx->hbox[b].nblocks; ++k) blk_box[ctx->hbox[b].block_begin + k] = b;
        for (int k = 0; k < 3; ++k) dyn[b].g[k] = dyn[nbox + b].g[k] = (float)boxes[b].body_force[k];
        dyn[b].eps = dyn[nbox + b].eps = 0.0f;
    }
    cudaError_t err = cudaSuccess;
    err = err ? err : cudaMemsetAsync(ctx->fbuf[0], 0, (size_t)off * ctx->elem, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->fbuf[1], 0, (size_t)off * ctx->elem, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_acc, 0, sizeof(long long) * NACC * ctx->maxp, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_rows, 0, sizeof(uint64_t) * 2ull * MAXS * MAXS * ctx->maxp, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned) * 4, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_pk, 0, sizeof(PartK) * ctx->maxp, ctx->stream);
    err = err ? err : cudaMemcpyAsync(ctx->d_boxes, ctx->hbox.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice, ctx->stream);
    err = err ? err : cudaMemcpyAsync(ctx->d_blk_box, blk_box.data(), sizeof(int) * blk, cudaMemcpyHostToDevice, ctx->stream);
    err = err ? err : cudaMemcpyAsync(ctx->d_box_dyn, dyn.data(), sizeof(BoxDyn) * 2 * nbox, cudaMemcpyHostToDevice, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_box_done, 0, sizeof(int) * nbox, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_need_hdr, 0, sizeof(NeedHdr) * 2 * (size_t)ctx->maxp, ctx->stream);
    err = err ? err : cudaMemsetAsync(ctx->d_need, 0, sizeof(uint64_t) * 2 * (size_t)MAXS * MAXS * ctx->maxp, ctx->stream);
    // the step kernel's counters start at zero and every launch leaves them so
    err = err ? err : cudaMemsetAsync(ctx->d_sync, 0, sizeof(unsigned) * (SYNC_HDR + (size_t)ctx->maxp + 2 * 4096), ctx->stream);
    err = err ? err : cudaStreamSynchronize(ctx->stream);
    if (err != cudaSuccess) {
        free_all(ctx);
        cudaStreamDestroy(ctx->stream);
        cudaEventDestroy(ctx->ev_done);
        delete ctx;
        return LB_ECUDA;
    }
    *out = ctx;
    return LB_OK;
}

extern "C" lb_status lb_destroy(lb_ctx* ctx)
{
    if (!ctx) return LB_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaDeviceSynchronize();
    free_all(ctx);
    if (ctx->s27) cudaStreamDestroy(ctx->s27);
    if (ctx->ev27a) cudaEventDestroy(ctx->ev27a);
    if (ctx->ev27b) cudaEventDestroy(ctx->ev27b);
    cudaStreamDestroy(ctx->stream);
    cudaEventDestroy(ctx->ev_done);
    delete ctx;
    return LB_OK;
}

// the critical particle kernel of iteration t (buffer parity cur) writes the box
// terms that the bulk and boundary kernels of iteration t+1 (parity cur^1) read
static PParams particle_params(lb_ctx* ctx, int cur)
{
    PParams pp{};
    pp.pd = ctx->d_pd; pp.pk = ctx->d_pk; pp.acc = ctx->d_acc; pp.rows = ctx->d_rows;
    pp.boxes = ctx->d_boxes; pp.box_dyn = ctx->d_box_dyn + (size_t)(cur ^ 1) * ctx->desc.size();
    pp.pdyn = ctx->d_pdyn + (size_t)(cur ^ 1) * ctx->maxp;
    pp.box_done = ctx->d_box_done;
    pp.need_hdr = ctx->d_need_hdr + (size_t)(cur ^ 1) * ctx->maxp;
    pp.need = ctx->d_need + (size_t)(cur ^ 1) * MAXS * MAXS * ctx->maxp;
    pp.status = ctx->d_status; pp.ring = ctx->d_ring; pp.np = ctx->np; pp.init = 0;
    pp.didt_mode = ctx->opt.didt_mode;
    pp.smax = 2 * (ctx->opt.max_semi + CUBE_MARGIN) + 2;
    return pp;
}

// bounding cube of one particle: h = ceil(max semi) + CUBE_MARGIN, S = 2h + 2
static void cube_of(const lb_particle& p, int& h, int& S)
{
    const double m = std::max(p.semi[0], std::max(p.semi[1], p.semi[2]));
    h = (int)std::ceil(m) + CUBE_MARGIN;
    S = 2 * h + 2;
}

// Partners: particles of a box whose bounding cubes come within reach of each
// other this step or the next (|x_b - x_a| < (S_a + S_b)/2 + 3 along every axis,
// minimum image, positions of the same time); the relation the critical
// blocks evaluate each step, from the same doubles in the same order for both
// particles of a pair, so it is symmetric.
static bool partners(const double xlo[3], int Slo, const double xhi[3], int Shi, const lb_box_desc& d)
{
    const int L[3] = {d.nx, d.ny, d.nz};
    const bool per[3] = {true, d.walls == 0, true};
    const double reach = 0.5 * (double)(Slo + Shi) + 3.0;
    for (int k = 0; k < 3; ++k) {
        double v = xhi[k] - xlo[k];
        if (per[k]) v = v - (double)L[k] * std::floor(v / (double)L[k] + 0.5);
        if (!(std::fabs(v) < reach)) return false;
    }
    return true;
}

extern "C" lb_status lb_set_particles(lb_ctx* ctx, int32_t box, const lb_particle* p, int32_t n)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->stepped) return fail(ctx, LB_ESTATE, "particles can only be set before the first step");
    if (box < 0 || box >= (int)ctx->desc.size() || n < 0 || (n > 0 && !p)) return fail(ctx, LB_EINVAL, "bad box or particle array");
    if (ctx->lattice == 27) {
        CK(cudaSetDevice(ctx->device));
        return q27_set_particles(ctx, box, p, n);
    }
    const lb_box_desc& d = ctx->desc[box];
    int total = 0;
    for (int b = 0; b < (int)ctx->parts.size(); ++b) total += (b == box) ? n : (int)ctx->parts[b].size();
    if (total > ctx->maxp) return fail(ctx, LB_EINVAL, "more particles than lb_options.max_particles");
    for (int i = 0; i < n; ++i) {
        const lb_particle& q = p[i];
        for (int k = 0; k < 3; ++k)
            if (!(q.semi[k] > 0.0) || q.semi[k] > ctx->opt.max_semi)
                return fail(ctx, LB_EINVAL, "semi-axis must be in (0, max_semi]");
        const double qn = std::sqrt(q.q[0] * q.q[0] + q.q[1] * q.q[1] + q.q[2] * q.q[2] + q.q[3] * q.q[3]);
        if (std::fabs(qn - 1.0) > 1e-6) return fail(ctx, LB_EINVAL, "quaternion must be unit");
        if (!(q.density > 0.0)) return fail(ctx, LB_EINVAL, "density must be positive");
        int h, S;
        cube_of(q, h, S);
        if (S > d.nx || S > d.nz || S > d.ny) return fail(ctx, LB_EINVAL, "particle too large for the box");
        if (d.walls) {
            const int oy = (int)std::floor(q.x[1]) - h;
            if (q.x[1] - std::max(q.semi[0], std::max(q.semi[1], q.semi[2])) <= 0.5 ||
                q.x[1] + std::max(q.semi[0], std::max(q.semi[1], q.semi[2])) >= d.ny - 1.5 || oy + S < 0)
                return fail(ctx, LB_EINVAL, "particle touches a wall");
        }
    }
    // particles whose cubes reach each other (partners): the box must leave room
    // for both cubes side by side, and clusters are tracked over at most MAXPB
    // particles of a box
    {
        std::vector<int> cnt(n, 0);
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                int hi_, Si, hj_, Sj;
                cube_of(p[i], hi_, Si);
                cube_of(p[j], hj_, Sj);
                if (!partners(p[i].x, Si, p[j].x, Sj, d)) continue;
                if (Si + Sj + 2 > d.nx || Si + Sj + 2 > d.nz || (!d.walls && Si + Sj + 2 > d.ny))
                    return fail(ctx, LB_EINVAL, "box too small for two nearby particles' cubes");
                ++cnt[i];
                ++cnt[j];
            }
        for (int i = 0; i < n; ++i)
            if (cnt[i] > MAXNB) return fail(ctx, LB_ECAPACITY, "a particle has more than MAXNB neighbours in reach");
        if (n > MAXPB) return fail(ctx, LB_EINVAL, "at most 64 particles in a box");
    }
    ctx->parts[box].assign(p, p + n);
    // rebuild the global particle table, boxes in order
    std::vector<PartDev> pd;
    int idx = 0;
    for (int b = 0; b < (int)ctx->parts.size(); ++b) {
        ctx->hbox[b].pbeg = idx;
        ctx->hbox[b].pcnt = (int)ctx->parts[b].size();
        for (const lb_particle& q : ctx->parts[b]) {
            PartDev s{};
            for (int k = 0; k < 3; ++k) {
                s.semi[k] = q.semi[k]; s.x[k] = q.x[k]; s.U[k] = q.U[k]; s.W[k] = q.Omega[k];
                s.Fext[k] = q.F_ext[k]; s.Text[k] = q.T_ext[k];
            }
            const double qn = std::sqrt(q.q[0] * q.q[0] + q.q[1] * q.q[1] + q.q[2] * q.q[2] + q.q[3] * q.q[3]);
            for (int k = 0; k < 4; ++k) s.q[k] = q.q[k] / qn;
            s.density = q.density; s.B1 = q.B1; s.B2 = q.B2;
            const double a = q.semi[0], bb = q.semi[1], c = q.semi[2];
            s.M = q.density * 4.0 / 3.0 * M_PI * a * bb * c;
            s.Ib[0] = s.M * (bb * bb + c * c) / 5.0;
            s.Ib[1] = s.M * (a * a + c * c) / 5.0;
            s.Ib[2] = s.M * (a * a + bb * bb) / 5.0;
            cube_of(q, s.h, s.S);
            s.box = b;
            s.aux_step = -1;
            s.lsum_step = -1;
            pd.push_back(s);
            ++idx;
        }
    }
    ctx->np = idx;
    CK(cudaSetDevice(ctx->device));
    if (idx > 0) CK(cudaMemcpyAsync(ctx->d_pd, pd.data(), sizeof(PartDev) * idx, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_boxes, ctx->hbox.data(), sizeof(BoxDev) * ctx->hbox.size(), cudaMemcpyHostToDevice, ctx->stream));
    // the snapshot's constant fields: squirmer parameters and the particle's box
    {
        std::vector<PartK> pk(ctx->maxp);
        std::memset(pk.data(), 0, sizeof(PartK) * pk.size());
        for (int i = 0; i < idx; ++i) {
            const PartDev& s = pd[i];
            const BoxDev& h = ctx->hbox[s.box];
            PartK& k = pk[i];
            k.box = s.box;
            k.a = (float)s.semi[0];
            k.b = (float)s.semi[1];
            k.eps2 = (float)std::fmax(0.0, 1.0 - (s.semi[1] * s.semi[1]) / (s.semi[0] * s.semi[0]));
            k.B1 = (float)s.B1;
            k.B2 = (float)s.B2;
            k.squirmer = (s.B1 != 0.0 || s.B2 != 0.0) ? 1 : 0;
            k.N = h.N; k.off = h.off; k.nwall = h.nwall; k.rho0 = h.rho0;
            k.nx = h.nx; k.ny = h.ny; k.nz = h.nz; k.walls = h.walls;
            k.omega = h.omega; k.rho0f = h.rho0f; k.scale = h.scale; k.inv_scale = h.inv_scale;
            for (int a = 0; a < 3; ++a) {
                k.uw_lo[a] = h.uw_lo[a]; k.uw_hi[a] = h.uw_hi[a];
                k.body[a] = (float)h.body[a];
            }
            k.counter = h.counter;
            k.pbeg = h.pbeg; k.pcnt = h.pcnt;
            k.lub_cut = h.lub_cut;
            k.mu = h.mu;
            k.nnb = 0;
            const lb_box_desc& bd = ctx->desc[s.box];
            for (int j = h.pbeg; j < h.pbeg + h.pcnt; ++j) {
                if (j == i) continue;
                const int lo = std::min(i, j), hi = std::max(i, j);
                if (partners(pd[lo].x, pd[lo].S, pd[hi].x, pd[hi].S, bd) && k.nnb < MAXNB) k.nb[k.nnb++] = j;
            }
        }
        std::vector<double> ring(2 * RINGD * (size_t)ctx->maxp, 0.0);
        for (int i = 0; i < idx; ++i)
            for (int t = 0; t < 2; ++t) {
                double* r = &ring[((size_t)i * 2 + t) * RINGD];
                for (int a = 0; a < 3; ++a) { r[a] = pd[i].x[a]; r[3 + a] = pd[i].U[a]; }
                for (int a = 0; a < 4; ++a) r[6 + a] = pd[i].q[a];
            }
        CK(cudaMemcpyAsync(ctx->d_ring, ring.data(), sizeof(double) * ring.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_pk, pk.data(), sizeof(PartK) * ctx->maxp, cudaMemcpyHostToDevice, ctx->stream));
        const size_t nb = ctx->desc.size();
        std::vector<BoxDyn> dyn(2 * nb), pdyn(2 * (size_t)ctx->maxp);
        for (size_t b = 0; b < nb; ++b) {
            for (int k = 0; k < 3; ++k) dyn[b].g[k] = dyn[nb + b].g[k] = (float)ctx->desc[b].body_force[k];
            dyn[b].eps = dyn[nb + b].eps = 0.0f;
        }
        for (int i = 0; i < idx; ++i) pdyn[i] = pdyn[ctx->maxp + i] = dyn[pd[i].box];
        CK(cudaMemcpyAsync(ctx->d_box_dyn, dyn.data(), sizeof(BoxDyn) * dyn.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_pdyn, pdyn.data(), sizeof(BoxDyn) * pdyn.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(ctx->d_box_done, 0, sizeof(int) * nb, ctx->stream));
        CK(cudaMemsetAsync(ctx->d_acc, 0, sizeof(long long) * NACC * ctx->maxp, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));     // the host vectors above go out of scope
    }
    clear_stale_error();
    // the initial state serves the first iteration, which reads parity ctx->cur
    PParams pp = particle_params(ctx, ctx->cur ^ 1);
    pp.init = 1;
    CK(launch_particles(pp, ctx->stream));
    CK(launch_particles_aux(pp, ctx->stream));
    CK(cudaEventRecord(ctx->ev_done, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
}

extern "C" lb_status lb_set_external(lb_ctx* ctx, int32_t box, const double* ft, int32_t n, void* stream)
{
    if (!ctx) return LB_EINVAL;
    const bool all = box == -1;
    if ((!all && (box < 0 || box >= (int)ctx->desc.size())) || !ft ||
        n != (all ? ctx->np : (int)ctx->parts[box].size()))
        return fail(ctx, LB_EINVAL, "bad box or count");
    if (n == 0) return LB_OK;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    if (ctx->lattice == 27) {
        // F_ext, T_ext are adjacent in the particle state; then the counter force
        const int slot = all ? 0 : ctx->box27_part[box];
        CK(cudaMemcpy2DAsync(&ctx->d_part27[slot].Fext[0], sizeof(q27::Part27), ft, 6 * sizeof(double),
                             6 * sizeof(double), n, cudaMemcpyHostToDevice, s));
        CK(q27::launch_refresh27(ctx->d_part27, ctx->d_box27, ctx->d_dyn27 + (size_t)ctx->dpar27 * ctx->desc.size(),
                                 ctx->np, s));
        return LB_OK;
    }
    const int pbeg = all ? 0 : ctx->hbox[box].pbeg;
    // one strided copy straight into the particle states (F_ext, T_ext are adjacent)
    CK(cudaMemcpy2DAsync(&ctx->d_pd[pbeg].Fext[0], sizeof(PartDev), ft, 6 * sizeof(double), 6 * sizeof(double), n,
                         cudaMemcpyHostToDevice, s));
    return LB_OK;
}

static KParams base_kparams(lb_ctx* ctx)
{
    KParams k{};
    k.boxes = ctx->d_boxes;
    k.nbox = (int)ctx->hbox.size();
    k.pk = ctx->d_pk;
    k.status = ctx->d_status;
    return k;
}

static BulkParams bulk_params(lb_ctx* ctx, int first, int cur)
{
    BulkParams bp{};
    bp.boxes = ctx->d_boxes; bp.blk_box = ctx->d_blk_box;
    bp.box_dyn = ctx->d_box_dyn + (size_t)cur * ctx->desc.size();
    bp.need_hdr = ctx->d_need_hdr + (size_t)cur * ctx->maxp;
    bp.need = ctx->d_need + (size_t)cur * MAXS * MAXS * ctx->maxp;
    bp.src = ctx->fbuf[cur]; bp.dst = ctx->fbuf[cur ^ 1]; bp.first = first;
    return bp;
}

static BndParams bnd_params(lb_ctx* ctx, int first, int cur)
{
    BndParams np{};
    np.pdyn = ctx->d_pdyn + (size_t)cur * ctx->maxp;
    np.pk = ctx->d_pk; np.acc = ctx->d_acc; np.rows = ctx->d_rows;
    np.need = ctx->d_need + (size_t)cur * MAXS * MAXS * ctx->maxp;
    np.need_hdr = ctx->d_need_hdr + (size_t)cur * ctx->maxp;
    np.status = ctx->d_status;
    np.src = ctx->fbuf[cur]; np.dst = ctx->fbuf[cur ^ 1];
    np.list_cap = ctx->list_cap; np.first = first;
    np.smax = 2 * (ctx->opt.max_semi + CUBE_MARGIN) + 2;
    np.gx = ctx->gx;
    return np;
}

// The auxiliary particle blocks left over by the last step-kernel launch (its
// last iteration's), before anything that reads their results.
static cudaError_t flush_aux(lb_ctx* ctx, cudaStream_t s)
{
    if (!ctx->aux_pending || ctx->np == 0) return cudaSuccess;
    const cudaError_t e = launch_particles_aux(particle_params(ctx, ctx->cur), s);
    if (e == cudaSuccess) ctx->aux_pending = false;
    return e;
}

// One iteration as separate kernels, in stream order on s.
static cudaError_t enqueue_iteration(lb_ctx* ctx, int first, int cur, cudaStream_t s)
{
    cudaError_t e;
    if ((e = flush_aux(ctx, s)) != cudaSuccess) return e;
    if ((e = launch_bulk(bulk_params(ctx, first, cur), ctx->kprec, ctx->total_blocks, s)) != cudaSuccess) return e;
    if (ctx->np == 0) return cudaSuccess;
    if ((e = launch_boundary(bnd_params(ctx, first, cur), ctx->kprec, ctx->np, s)) != cudaSuccess) return e;
    const PParams pp = particle_params(ctx, cur);
    if ((e = launch_particles(pp, s)) != cudaSuccess) return e;
    return launch_particles_aux(pp, s);
}

// k iterations in one launch of the step kernel, starting at buffer parity cur;
// io_ft / io_rec (device-accessible, or null): per-iteration external forces
// in and particle records out
static cudaError_t enqueue_steps(lb_ctx* ctx, int k, int cur, cudaStream_t s, const double* io_ft = nullptr,
                                 double* io_rec = nullptr)
{
    BulkParams bulk[2];
    BndParams bnd[2];
    PParams part[2];
    for (int c = 0; c < 2; ++c) {
        bulk[c] = bulk_params(ctx, 0, c);
        bnd[c] = bnd_params(ctx, 0, c);
        part[c] = particle_params(ctx, c);
    }
    // no reset of the counters: each launch leaves them at zero
    const cudaError_t e = launch_step(bulk, bnd, part, ctx->d_sync, ctx->d_status, ctx->np, ctx->gx, ctx->total_blocks,
                                      k, cur, ctx->kprec, ctx->fetch, io_ft, io_rec, s);
    if (e == cudaSuccess && ctx->np > 0) ctx->aux_pending = true;
    return e;
}

// A stream that is being captured into a CUDA graph: its work is recorded,
// not run, so the context's completion event is neither waited on nor
// recorded there (an event recorded inside a capture cannot be waited on
// outside it).
static bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

extern "C" lb_status lb_step(lb_ctx* ctx, int32_t nsteps, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (nsteps < 0) return fail(ctx, LB_EINVAL, "negative step count");
    if (nsteps == 0) return LB_OK;
    CK(cudaSetDevice(ctx->device));
    clear_stale_error();
    cudaStream_t s = pick(ctx, stream);
    const bool cap = capturing(s);
    if (!cap && ctx->last_user_stream && ctx->last_user_stream != s) CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    ctx->last_user_stream = s;
    ctx->stepped = true;
    if (ctx->lattice == 27) {
        CK(q27_enqueue(ctx, nsteps, s));
        if (!cap) CK(cudaEventRecord(ctx->ev_done, s));
        return LB_OK;
    }
    int left = nsteps;
    if (!ctx->collided) {
        CK(enqueue_iteration(ctx, 1, ctx->cur, s));
        ctx->cur ^= 1;
        ctx->collided = true;
        --left;
    }
    const bool separate = (ctx->opt.flags & LB_FLAG_SEPARATE_KERNELS) != 0;
    while (left > 0) {
        if (separate) {
            CK(enqueue_iteration(ctx, 0, ctx->cur, s));
            ctx->cur ^= 1;
            --left;
        } else {
            const int k = left < STEP_ITERS ? left : STEP_ITERS;
            CK(enqueue_steps(ctx, k, ctx->cur, s));
            ctx->cur ^= (k & 1);
            left -= k;
        }
    }
    if (!cap) CK(cudaEventRecord(ctx->ev_done, s));
    return LB_OK;
}

extern "C" lb_status lb_profile_step(lb_ctx* ctx, int32_t nsteps, void* stream, double* ms_out)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    if (nsteps <= 0 || !ms_out) return fail(ctx, LB_EINVAL, "bad step count or output");
    CK(cudaSetDevice(ctx->device));
    clear_stale_error();
    cudaStream_t s = pick(ctx, stream);
    if (ctx->last_user_stream && ctx->last_user_stream != s) CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    ctx->last_user_stream = s;
    ctx->stepped = true;
    CK(flush_aux(ctx, s));
    cudaEvent_t ev[5];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double t[4] = {0, 0, 0, 0};
    for (int i = 0; i < nsteps; ++i) {
        const int first = ctx->collided ? 0 : 1;
        const BulkParams bp = bulk_params(ctx, first, ctx->cur);
        const BndParams np = bnd_params(ctx, first, ctx->cur);
        const PParams pp = particle_params(ctx, ctx->cur);
        CK(cudaEventRecord(ev[0], s));
        CK(launch_bulk(bp, ctx->kprec, ctx->total_blocks, s));
        CK(cudaEventRecord(ev[1], s));
        CK(launch_boundary(np, ctx->kprec, ctx->np, s));
        CK(cudaEventRecord(ev[2], s));
        CK(launch_particles(pp, s));
        CK(cudaEventRecord(ev[3], s));
        CK(launch_particles_aux(pp, s));
        CK(cudaEventRecord(ev[4], s));
        CK(cudaEventSynchronize(ev[4]));
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            t[k] += ms;
        }
        ctx->cur ^= 1;
        ctx->collided = true;
    }
    CK(cudaEventRecord(ctx->ev_done, s));
    for (auto& e : ev) cudaEventDestroy(e);
    ms_out[0] = t[0];            // bulk
    ms_out[1] = t[1];            // boundary
    ms_out[2] = t[2];            // particle critical
    ms_out[3] = t[3];            // particle auxiliary
    return read_status(ctx);
}

extern "C" lb_status lb_synchronize(lb_ctx* ctx)
{
    if (!ctx) return LB_EINVAL;
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    return read_status(ctx);
}

extern "C" lb_status lb_get_fields(lb_ctx* ctx, int32_t box, uint32_t what, void* dst, size_t dst_bytes,
                                   int32_t dst_is_device, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (box < 0 || box >= (int)ctx->desc.size() || !dst) return fail(ctx, LB_EINVAL, "bad box or destination");
    if (ctx->lattice == 27) {
        CK(cudaSetDevice(ctx->device));
        return q27_get_fields(ctx, box, what, dst, dst_bytes, dst_is_device, pick(ctx, stream));
    }
    const BoxDev& B = ctx->hbox[box];
    size_t need = 0;
    switch (what) {
    case LB_FIELD_F: case LB_FIELD_DF: need = 19ull * B.N * 4; break;
    case LB_FIELD_RHO: case LB_FIELD_SOLID: need = (size_t)B.N * 4; break;
    case LB_FIELD_U: need = 3ull * B.N * 4; break;
    default: return fail(ctx, LB_EINVAL, "exactly one LB_FIELD_* bit");
    }
    if (dst_bytes != need) return fail(ctx, LB_EINVAL, "dst_bytes does not match the field size");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    const bool direct = dst_is_device && ((uintptr_t)dst % 16 == 0);
    if (!direct && !ctx->d_tmp) {
        ctx->d_tmp = (float*)dev_alloc(ctx, ctx->tmp_bytes);
        if (!ctx->d_tmp) return fail(ctx, LB_ENOMEM, "field staging buffer");
    }
    float* out = direct ? (float*)dst : ctx->d_tmp;
    KParams k = base_kparams(ctx);
    k.src = ctx->fbuf[ctx->cur];
    k.only_box = box;
    k.nopull = ctx->collided ? 0 : 1;
    k.out_dev = (what == LB_FIELD_DF) ? 1 : 0;
    if (what == LB_FIELD_F || what == LB_FIELD_DF) k.out_f = out;
    if (what == LB_FIELD_RHO) k.out_rho = out;
    if (what == LB_FIELD_U) k.out_u = out;
    if (what == LB_FIELD_SOLID) k.out_solid = (int*)out;
    CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    CK(launch_fields(k, ctx->opt.precision, B.nblocks, s));
    if (!direct) CK(cudaMemcpyAsync(dst, out, need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return read_status(ctx);
}

extern "C" lb_status lb_get_force_torque(lb_ctx* ctx, int32_t box, double* out, int32_t n)
{
    if (!ctx) return LB_EINVAL;
    const bool all = box == -1;
    if ((!all && (box < 0 || box >= (int)ctx->desc.size())) || !out ||
        n != (all ? ctx->np : (int)ctx->parts[box].size()))
        return fail(ctx, LB_EINVAL, "bad box, buffer or count");
    if (n == 0) return LB_OK;
    CK(cudaSetDevice(ctx->device));
    if (ctx->last_user_stream) CK(cudaStreamSynchronize(ctx->last_user_stream));
    if (ctx->lattice == 27) {
        const int slot = all ? 0 : ctx->box27_part[box];
        CK(cudaMemcpy2DAsync(out, sizeof(double) * LB_RECORD_DOUBLES, &ctx->d_part27[slot].rec[0], sizeof(q27::Part27),
                             sizeof(double) * LB_RECORD_DOUBLES, n, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return read_status(ctx);
    }
    const int pbeg = all ? 0 : ctx->hbox[box].pbeg;
    // gather the records into one staging block, then a single copy
    if (!ctx->d_rec) {
        ctx->d_rec = (double*)dev_alloc(ctx, sizeof(double) * LB_RECORD_DOUBLES * ctx->maxp);
        if (!ctx->d_rec) return fail(ctx, LB_ENOMEM, "record staging buffer");
    }
    CK(cudaMemcpy2DAsync(ctx->d_rec, sizeof(double) * LB_RECORD_DOUBLES, &ctx->d_pd[pbeg].rec[0], sizeof(PartDev),
                         sizeof(double) * LB_RECORD_DOUBLES, n, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(out, ctx->d_rec, sizeof(double) * LB_RECORD_DOUBLES * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
}

extern "C" lb_status lb_get_force_torque_async(lb_ctx* ctx, int32_t box, double* out, int32_t n, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    const bool all = box == -1;
    if ((!all && (box < 0 || box >= (int)ctx->desc.size())) || !out ||
        n != (all ? ctx->np : (int)ctx->parts[box].size()))
        return fail(ctx, LB_EINVAL, "bad box, buffer or count");
    if (n == 0) return LB_OK;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    if (!capturing(s)) CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    const int pbeg = all ? 0 : ctx->hbox[box].pbeg;
    // one strided copy straight out of the particle states
    CK(cudaMemcpy2DAsync(out, sizeof(double) * LB_RECORD_DOUBLES, &ctx->d_pd[pbeg].rec[0], sizeof(PartDev),
                         sizeof(double) * LB_RECORD_DOUBLES, n, cudaMemcpyDefault, s));
    return LB_OK;
}

// Device address of caller memory of `bytes` bytes that the GPU of the
// context can read and write directly: its own device memory, managed memory,
// or page-locked host memory (through its mapped address; both ends of the
// range must lie in the same mapping).  Null when it cannot (pageable host
// memory, another GPU), and the caller then copies instead.
static void* device_view(lb_ctx* ctx, const void* p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a, b;
    const char* last = static_cast<const char*>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != b.type || !a.devicePointer || !b.devicePointer) return nullptr;
    if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->device) return nullptr;
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged && a.type != cudaMemoryTypeHost) return nullptr;
    return a.devicePointer;
}

extern "C" lb_status lb_step_io(lb_ctx* ctx, int32_t nsteps, const double* ft, double* rec, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    if (nsteps < 0) return fail(ctx, LB_EINVAL, "negative step count");
    if (nsteps == 0) return LB_OK;
    const size_t np = (size_t)ctx->np;
    if (np == 0 || (!ft && !rec)) return lb_step(ctx, nsteps, stream);
    CK(cudaSetDevice(ctx->device));
    const double* dft = static_cast<const double*>(device_view(ctx, ft, sizeof(double) * 6 * np * nsteps));
    double* drec = static_cast<double*>(device_view(ctx, rec, sizeof(double) * RECD * np * nsteps));
    // the step kernel reads F_ext / T_ext and writes the records itself when
    // the GPU can reach the caller's memory (on GB300, page-locked host memory
    // over the coherent CPU-GPU link); otherwise, and for the first collision
    // and in the separate-kernel mode, three queued calls per step
    const bool direct = !(ctx->opt.flags & LB_FLAG_SEPARATE_KERNELS) && (!ft || dft) && (!rec || drec);
    int k = 0;
    while (k < nsteps && (!direct || !ctx->collided)) {
        lb_status r;
        if (ft && (r = lb_set_external(ctx, -1, ft + k * np * 6, ctx->np, stream)) != LB_OK) return r;
        if ((r = lb_step(ctx, 1, stream)) != LB_OK) return r;
        if (rec && (r = lb_get_force_torque_async(ctx, -1, rec + k * np * RECD, ctx->np, stream)) != LB_OK) return r;
        ++k;
    }
    if (k == nsteps) return LB_OK;
    clear_stale_error();
    cudaStream_t s = pick(ctx, stream);
    const bool cap = capturing(s);
    if (!cap && ctx->last_user_stream && ctx->last_user_stream != s) CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    ctx->last_user_stream = s;
    ctx->stepped = true;
    while (k < nsteps) {
        const int c = nsteps - k < STEP_ITERS ? nsteps - k : STEP_ITERS;
        CK(enqueue_steps(ctx, c, ctx->cur, s, dft ? dft + k * np * 6 : nullptr, drec ? drec + k * np * RECD : nullptr));
        ctx->cur ^= (c & 1);
        k += c;
    }
    if (!cap) CK(cudaEventRecord(ctx->ev_done, s));
    return LB_OK;
}

extern "C" lb_status lb_get_drag(lb_ctx* ctx, int32_t box, int32_t particle, double* out36)
{
    if (!ctx) return LB_EINVAL;
    if (box < 0 || box >= (int)ctx->desc.size() || particle < 0 || particle >= (int)ctx->parts[box].size() || !out36)
        return fail(ctx, LB_EINVAL, "bad box or particle");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    if (ctx->lattice == 27) {
        CK(cudaMemcpy(out36, &ctx->d_part27[ctx->box27_part[box]].zeta[0], 36 * sizeof(double), cudaMemcpyDeviceToHost));
        return read_status(ctx);
    }
    CK(flush_aux(ctx, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(out36, &ctx->d_pd[ctx->hbox[box].pbeg + particle].zeta[0], 36 * sizeof(double), cudaMemcpyDeviceToHost));
    return read_status(ctx);
}

extern "C" lb_status lb_get_links(lb_ctx* ctx, int32_t box, int32_t particle, int32_t* pairs, int32_t cap,
                                  int32_t* count)
{
    if (!ctx) return LB_EINVAL;
    if (box < 0 || box >= (int)ctx->desc.size() || particle < 0 || particle >= (int)ctx->parts[box].size() ||
        !count || cap < 0 || (cap > 0 && !pairs))
        return fail(ctx, LB_EINVAL, "bad box, particle or buffer");
    CK(cudaSetDevice(ctx->device));
    if (!ctx->d_links) {
        ctx->links_cap = MAXS * MAXS * (ctx->lattice == 27 ? 26 : 18);
        ctx->d_links = (int*)dev_alloc(ctx, sizeof(int) * 2ull * ctx->links_cap);
        if (!ctx->d_links) return fail(ctx, LB_ENOMEM, "link buffer");
    }
    CK(cudaDeviceSynchronize());
    if (ctx->lattice == 27) {
        CK(cudaMemsetAsync(ctx->d_count, 0, sizeof(int), ctx->stream));
        CK(q27::launch_links27(ctx->d_part27, ctx->d_box27, ctx->d_rows, ctx->box27_part[box], ctx->d_links,
                               ctx->links_cap, ctx->d_count, ctx->stream));
    } else {
        const int p = ctx->hbox[box].pbeg + particle;
        CK(launch_links(ctx->d_pd, ctx->d_pk, ctx->d_rows, ctx->d_boxes, p, ctx->d_links, ctx->links_cap, ctx->d_count,
                        ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    int n = 0;
    CK(cudaMemcpy(&n, ctx->d_count, sizeof(int), cudaMemcpyDeviceToHost));
    *count = n;
    if (n <= cap && n > 0) CK(cudaMemcpy(pairs, ctx->d_links, sizeof(int) * 2ull * n, cudaMemcpyDeviceToHost));
    return read_status(ctx);
}

// ---------------------------------------------------------------------------
// Warm start: an initial fluid field and the periodic Stokes flow of the
// particles' forces (warm_kernel.cu).

// owner field of box `box` into d_tmp[0, N) (before the first collision)
static cudaError_t owner_field(lb_ctx* ctx, int box, cudaStream_t s)
{
    KParams k = base_kparams(ctx);
    k.src = ctx->fbuf[ctx->cur];
    k.only_box = box;
    k.nopull = 1;
    k.out_solid = reinterpret_cast<int*>(ctx->d_tmp);
    return launch_fields(k, ctx->opt.precision, ctx->hbox[box].nblocks, s);
}

extern "C" lb_status lb_init_fluid(lb_ctx* ctx, int32_t box, const float* u, size_t u_bytes, const float* drho,
                                   int32_t is_device, int32_t with_stress, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    if (box < 0 || box >= (int)ctx->desc.size() || !u) return fail(ctx, LB_EINVAL, "bad box or field");
    if (ctx->stepped) return fail(ctx, LB_ESTATE, "lb_init_fluid after the first step");
    const BoxDev& B = ctx->hbox[box];
    if (u_bytes != 3ull * B.N * sizeof(float)) return fail(ctx, LB_EINVAL, "u_bytes must be 3*N*4");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    if (!ctx->d_tmp) {
        ctx->d_tmp = (float*)dev_alloc(ctx, ctx->tmp_bytes);
        if (!ctx->d_tmp) return fail(ctx, LB_ENOMEM, "field staging buffer");
    }
    float* ud = ctx->d_tmp + B.N;                      // [3][N] after the owner field, then drho [N]
    float* dd = drho ? ctx->d_tmp + 4 * B.N : nullptr;
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    CK(cudaMemcpyAsync(ud, u, u_bytes, kind, s));
    if (dd) CK(cudaMemcpyAsync(dd, drho, (size_t)B.N * sizeof(float), kind, s));
    CK(owner_field(ctx, box, s));
    CK(launch_init_fluid(B, ctx->opt.precision, ctx->fbuf[ctx->cur], ud, dd, reinterpret_cast<int*>(ctx->d_tmp),
                         (float)ctx->desc[box].tau, with_stress != 0, s));
    CK(cudaStreamSynchronize(s));
    return read_status(ctx);
}

extern "C" lb_status lb_stokes_field(lb_ctx* ctx, int32_t box, float* u_dev, float* drho_dev, void* stream)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    if (box < 0 || box >= (int)ctx->desc.size() || !u_dev) return fail(ctx, LB_EINVAL, "bad box or output");
    const lb_box_desc& d = ctx->desc[box];
    if (d.walls) return fail(ctx, LB_EINVAL, "lb_stokes_field needs a fully periodic box");
    if (d.nx > 4096 || d.ny > 4096 || d.nz > 4096) return fail(ctx, LB_EINVAL, "box edge above 4096");
    if (ctx->stepped) return fail(ctx, LB_ESTATE, "lb_stokes_field after the first step");
    const BoxDev& B = ctx->hbox[box];
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    if (!ctx->d_tmp) {
        ctx->d_tmp = (float*)dev_alloc(ctx, ctx->tmp_bytes);
        if (!ctx->d_tmp) return fail(ctx, LB_ENOMEM, "field staging buffer");
    }
    if (!ctx->d_stokes) {
        long long nmax = 0;
        for (auto& h : ctx->hbox) nmax = std::max(nmax, h.N);
        ctx->d_stokes = (float2*)dev_alloc(ctx, sizeof(float2) * 8 * (size_t)nmax);
        // np + 1 counts, then (8-byte aligned) 4 double sums
        ctx->d_counts = (int*)dev_alloc(ctx, sizeof(double) * ((size_t)(ctx->maxp + 2) / 2 + 4));
        if (!ctx->d_stokes || !ctx->d_counts) return fail(ctx, LB_ENOMEM, "Stokes work buffers");
    }
    CK(cudaStreamWaitEvent(s, ctx->ev_done, 0));
    CK(owner_field(ctx, box, s));
    float* out = ctx->d_tmp + B.N;                     // [4][N]: u, then drho
    CK(launch_stokes(B, reinterpret_cast<int*>(ctx->d_tmp), ctx->d_pd + B.pbeg, B.pcnt, d.counter_force,
                     d.body_force, ctx->d_stokes, ctx->d_counts,
                     reinterpret_cast<double*>(ctx->d_counts) + (ctx->maxp + 2) / 2, out, s));
    CK(cudaMemcpyAsync(u_dev, out, 3ull * B.N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (drho_dev) CK(cudaMemcpyAsync(drho_dev, out + 3 * B.N, (size_t)B.N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return read_status(ctx);
}

// ---------------------------------------------------------------------------
// Autotuner of the step kernel's launch shape on the context's own boxes:
// first the number of blocks that share a particle's boundary nodes (gx: 1,
// 2, 3 or the size-based default; fewer blocks spend less SM time on fixed
// per-block costs, more blocks shorten the particle chain), then how many
// consecutive 32-quad bulk units a warp takes per fetch from the work counter
// (1, 2, 4, 8).  Every candidate computes the same values bit for bit: the
// boundary sums are integer atomics, whose order does not matter, and the
// assignment of bulk units to warps does not enter any node's arithmetic.
static int list_cap_for(lb_ctx* ctx, int gx)
{
    const long long Smax = 2ll * (ctx->opt.max_semi + CUBE_MARGIN) + 2;
    const long long total = std::min(Smax * Smax * Smax, 16 * Smax * Smax);
    return (int)((total + gx - 1) / gx);
}

extern "C" lb_status lb_autotune(lb_ctx* ctx, int32_t steps_per_candidate, void* stream, int32_t* out3,
                                 double* ms_per_step)
{
    if (!ctx) return LB_EINVAL;
    if (ctx->lattice == 27) return fail(ctx, LB_ESTATE, "not available with the D3Q27 lattice");
    if (steps_per_candidate < 1) return fail(ctx, LB_EINVAL, "steps_per_candidate must be positive");
    if (ctx->opt.flags & LB_FLAG_SEPARATE_KERNELS) return fail(ctx, LB_ESTATE, "no step kernel to tune");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = pick(ctx, stream);
    int advanced = 0;
    if (!ctx->collided) {
        const lb_status r = lb_step(ctx, 1, stream);
        if (r != LB_OK) return r;
        advanced = 1;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timed = [&](double& per) -> lb_status {
        lb_status r = lb_step(ctx, 2, stream);              // warm the new shape
        if (r != LB_OK) return r;
        CK(cudaEventRecord(e0, s));
        r = lb_step(ctx, steps_per_candidate, stream);
        if (r != LB_OK) return r;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        per = ms / steps_per_candidate;
        advanced += 2 + steps_per_candidate;
        return LB_OK;
    };
    const long long Smax = 2ll * (ctx->opt.max_semi + CUBE_MARGIN) + 2;
    const int gx0 = (int)std::max(1ll, (3 * Smax * Smax + BBLOCK - 1) / BBLOCK);
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    // fewer blocks than the size-based default leave more SMs to the bulk work;
    // more shorten the chain boundary -> critical block, which an iteration of
    // 16-bit storage can wait for
    const int gcand[6] = {1, 2, 3, gx0, 2 * gx0, 3 * gx0};
    double best = 1e300;
    int best_gx = ctx->gx;
    for (int c = 0; c < 6; ++c) {
        if (ms_per_step) ms_per_step[c] = 0.0;
        if (ctx->np == 0 || (c < 3 && gcand[c] >= gx0)) continue;    // below the default only
        // a boundary block gives one thread to each of its cube rows: the blocks
        // of a particle must have a thread for every one of its S^2 rows
        if ((long long)gcand[c] * BBLOCK < Smax * Smax) continue;
        if (c > 3 && (long long)ctx->np * (gcand[c] + 1) > 2ll * nsm) continue;   // one block per particle item
        // the node list of one block lives in shared memory next to two maps
        const size_t smem = 2ull * Smax * Smax * sizeof(uint64_t) + (size_t)list_cap_for(ctx, gcand[c]) * 4;
        if (smem > 100 * 1024) continue;
        ctx->gx = gcand[c];
        ctx->list_cap = list_cap_for(ctx, gcand[c]);
        double per = 0.0;
        const lb_status r = timed(per);
        if (r != LB_OK) return r;
        if (ms_per_step) ms_per_step[c] = per;
        if (per < best) { best = per; best_gx = gcand[c]; }
    }
    ctx->gx = best_gx;
    ctx->list_cap = list_cap_for(ctx, best_gx);
    static const int fcand[4] = {1, 2, 4, 8};
    best = 1e300;
    int best_f = ctx->fetch;
    for (int c = 0; c < 4; ++c) {
        ctx->fetch = fcand[c];
        double per = 0.0;
        const lb_status r = timed(per);
        if (r != LB_OK) return r;
        if (ms_per_step) ms_per_step[6 + c] = per;
        if (per < best) { best = per; best_f = fcand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->fetch = best_f;
    if (out3) {
        out3[0] = best_f;
        out3[1] = best_gx;
        out3[2] = advanced;
    }
    return read_status(ctx);
}
