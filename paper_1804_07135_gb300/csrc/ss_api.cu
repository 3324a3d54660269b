// ss_api.cu -- host runtime of libss: contexts, size groups, device buffers, the dipole-tensor
// spectrum, launch configuration, CUDA-graph replay of the iteration, and the C ABI of ss.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ss.h"
#include "ss_fft.cuh"
#include "ss_internal.h"

using namespace ss;

namespace {

thread_local std::string g_create_error;

// ---- small helpers --------------------------------------------------------------------------------
bool is_smooth23(int m) {
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

// Padded transform length: the smallest 2^a 3^b >= 2n - 1, enough for the linear (non-circular)
// convolution of n sites with offsets -(n-1)..(n-1) (Sec. II-A, the zero-padded kernel).
// Padded transform length for n sites: the smallest 2^a 3^b >= 2n - 1, or the power of two >= 2n - 1
// when that is at most 1/8 longer (its transforms need no radix-3 stages: 112 sites pad to 256, not 243).
int padded_len(int n) {
    int m = std::max(1, 2 * n - 1);
    while (!is_smooth23(m)) ++m;
    int p2 = 1;
    while (p2 < 2 * n - 1) p2 <<= 1;
    return 8 * p2 <= 9 * m ? p2 : m;
}

FftPlan make_plan(int P) { return fft_make_plan(P); }

// Eq. 7 at an integer lattice offset (entries xx, yy, zz, xy, xz, yz), with its 1/(4 pi).
void dipole_tensor_at(int dx, int dy, int dz, double out[6]) {
    const double x = dx, y = dy, z = dz;
    const double r2 = x * x + y * y + z * z;
    const double r = sqrt(r2);
    const double inv3 = 1.0 / (r2 * r), inv5 = inv3 / r2;
    const double c = 0.25 / M_PI;
    out[0] = c * (3.0 * x * x * inv5 - inv3);
    out[1] = c * (3.0 * y * y * inv5 - inv3);
    out[2] = c * (3.0 * z * z * inv5 - inv3);
    out[3] = c * 3.0 * x * y * inv5;
    out[4] = c * 3.0 * x * z * inv5;
    out[5] = c * 3.0 * y * z * inv5;
}

// exp(-2 pi i k / P), k = 0..P-1, in FP64.
std::vector<double2> twiddles(int P) {
    std::vector<double2> w(P);
    for (int k = 0; k < P; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)P;
        w[k] = make_double2(cos(a), -sin(a));
    }
    return w;
}


}  // namespace

// Twiddle tables of the two-pass transforms (layout in GroupArgs::t2x / t2y) of length P from the flat
// FP64 table w[k] = W_P^k; zeros when P is not a multiple of 16 (no two-pass transform then).
template <typename C> void two_pass_twiddles(int P, const std::vector<double2>& w, C* out) {
    using R = decltype(C{}.x);
    for (int i = 0; i < 2 * P; ++i) out[i] = C{R(0), R(0)};
    if (P % 16 != 0) return;
    const int R2 = P / 16;
    for (int e = 0; e < 16; ++e)  // e = 2m + par
        for (int n2 = 0; n2 < R2; ++n2) {
            const double2 x = w[(n2 * e) % P];
            out[e * R2 + n2] = C{R(x.x), R(x.y)};
        }
    for (int e = 0; e < R2; ++e)  // e = 2m + par2
        for (int k1 = 0; k1 < 16; ++k1) {
            const double2 x = w[(k1 * e) % P];
            out[P + e * 16 + k1] = C{R(x.x), R(x.y)};
        }
}

// ---- context --------------------------------------------------------------------------------------
struct Group {
    int rbytes = 4;  // bytes of the group's real type (4: the FP32 path, 8: FP64)
    // energy evaluations are cached per state: state_epoch advances whenever the group's path changes
    // (ss_set_path, ss_step, ss_time_kernels), eval_epoch records the state the FP64 energies are of
    long long state_epoch = 0, eval_epoch = -1;
    int nx = 0, ny = 0, nz = 0, N = 0, Px = 1, Py = 1;
    int n_img = 0, n_pairs = 0;
    std::vector<int> strs;  // context string ids, in group order
    std::vector<int> str_img0, str_K;
    bool dipole = false;  // FFT dipole convolution (SS_DIPOLE_FFT and some w != 0)
    bool direct = false;  // direct dipole sums (SS_DIPOLE_DIRECT and some w != 0)
    void* hdir = nullptr; // [image][3][N] direct sums
    FftPlan planx{}, plany{};
    int lsx = 1, lsy = 1;
    int ty_a = 1, ty_c = 1, thr_a = 128, thr_b = 128, thr_c = 128, thr_arc = 256;
    int yz_kxb = 0;  // kx columns per CTA of the two-pass y/z kernel (0: default; autotuned)
    size_t smem_a = 0, smem_b = 0, smem_c = 0, smem_c_eval = 0;
    int n_eblk = 0;
    // device
    void *s = nullptr, *sp = nullptr, *spec = nullptr, *dhat = nullptr, *twx = nullptr, *twy = nullptr;
    void *twxs = nullptr, *twys = nullptr;
    void *t2x = nullptr, *t2y = nullptr;  // two-pass twiddle tables (2 Px, 2 Py entries)
    void *prm = nullptr, *hout = nullptr;
    InterpEntry* interp = nullptr;
    double* epart = nullptr;
    int *d_str_img0 = nullptr, *d_str_K = nullptr;
    double *dpart = nullptr, *e_last = nullptr, *eval_terms = nullptr, *eval_E = nullptr, *eval_cn = nullptr;
    int* pair_on = nullptr;  // FP64 evaluation copy: the pairs holding barrier candidates
    // barrier candidates of an FP32 context (ss_barrier): the FP32 energies and round-off bounds select the
    // images whose FP64 energy can decide the barrier; their FP64 energies, valid for state bar_epoch
    long long bar_epoch = -1;
    std::vector<double> bar_E;  // [image] FP64 energy of a candidate, or NaN

    unsigned* arc_cnt = nullptr;
    // adaptive Runge-Kutta evolution (allocated by ss_set_integrator)
    void *rk_y0 = nullptr, *rk_k = nullptr, *rk_y5 = nullptr;
    double* rk_errp = nullptr;
    RkString* rk_st = nullptr;
    int *rk_img_sys = nullptr, *rk_sys_img0 = nullptr, *rk_sys_cnt = nullptr;
    int rk_nsys = 0;
    int* rk_active = nullptr;
    InterpEntry* interp_ident = nullptr;
    int rk_tiles = 0;
    // reparametrisation variants (allocated by ss_set_reparam)
    void* hc = nullptr;  // [image][3][N] force of the climbing image
    int* climb_img = nullptr;
    ArcArgs arc{};
};

struct StringRec {
    ss_string_desc d;
    int group;
    int local;  // index within its group
    int img0;   // first group-local image
    bool has_path;
};

struct ss_ctx {
    ss_opts opts{};
    int device = 0;
    std::vector<StringRec> strs;
    std::vector<Group> groups;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int* d_err = nullptr;
    void* stage = nullptr;  // device staging buffer for host copies
    size_t stage_bytes = 0;
    std::vector<std::pair<void*, size_t>> allocs;
    ss_alloc_fn alloc_fn = nullptr;  // the allocator the context was created with (null: cudaMalloc)
    ss_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    cudaGraphExec_t graph1 = nullptr, graphN = nullptr;
    cudaGraphExec_t rk_graph1 = nullptr, rk_graphN = nullptr;  // adaptive integrator: 1 and kRkGraphIters iterations
    cudaStream_t rk_body = nullptr;  // captures the bodies of the attempt-round WHILE nodes
    // several size groups: one graph branch per group (their strings never interact), forked from and
    // joined back into cs
    std::vector<cudaStream_t> branch;  // one per size group
    std::vector<cudaEvent_t> branch_ev;  // [0] fork, [1..] joins
    int graphN_iters = 64;
    int integrator = 0;  // SS_INT_EULER or one of the Runge-Kutta kinds
    int interp = 0;      // SS_INTERP_LINEAR or SS_INTERP_SPLINE
    int climb = 0;       // climbing image on
    int dynamics = 0;    // SS_DYN_STRING or SS_DYN_LLG
    double alpha = 0.0;  // damping of the precessional dynamics
    double rtol = 1e-6, atol = 1e-8;
    // FP32 contexts: an FP64 copy of every size group's evaluation pipeline, built on the first energy
    // query; reported energies and energy terms are evaluated there from the FP32 state
    std::vector<Group> ev64;
    std::string err;
};

namespace {

ss_status fail(ss_ctx* c, ss_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA,       \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Device memory of a context: from the allocator it was created with (ss_set_allocator), else cudaMalloc.
ss_status dalloc(ss_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->alloc_fn) {
        *p = c->alloc_fn(bytes, c->device, c->opts.stream, c->alloc_user);
        if (!*p) return fail(c, SS_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
        if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
            c->free_fn(*p, bytes, c->device, c->opts.stream, c->alloc_user);
            *p = nullptr;
            return fail(c, SS_ERR_INVALID_ARG, "allocator callback returned a pointer not aligned to 256 bytes");
        }
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            return fail(c, SS_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    c->allocs.push_back({*p, bytes});
    return SS_OK;
}

std::mutex g_alloc_mu;
ss_alloc_fn g_alloc_fn = nullptr;
ss_free_fn g_free_fn = nullptr;
void* g_alloc_user = nullptr;

#define TRY(x)                        \
    do {                              \
        ss_status s_ = (x);           \
        if (s_ != SS_OK) return s_;   \
    } while (0)

bool use_fp64(const ss_ctx* c) { return c->opts.precision == SS_PREC_FP64; }
size_t real_size(const ss_ctx* c) { return use_fp64(c) ? sizeof(double) : sizeof(float); }

template <typename T> GroupArgs<T> group_args(const ss_ctx* c, const Group& g) {
    GroupArgs<T> a{};
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.N = g.N;
    a.Px = g.Px;
    a.Py = g.Py;
    a.n_img = g.n_img;
    a.n_pairs = g.n_pairs;
    a.lsx = g.lsx;
    a.lsy = g.lsy;
    a.s = (T*)g.s;
    a.sp = (T*)g.sp;
    a.spec = (cplx<T>*)g.spec;
    a.dhat = (const T*)g.dhat;
    a.twx = (const cplx<T>*)g.twx;
    a.twy = (const cplx<T>*)g.twy;
    a.twxs = (const cplx<T>*)g.twxs;
    a.twys = (const cplx<T>*)g.twys;
    a.t2x = (const cplx<T>*)g.t2x;
    a.t2y = (const cplx<T>*)g.t2y;
    a.planx = g.planx;
    a.plany = g.plany;
    a.prm = (const ImgParam<T>*)g.prm;
    a.interp = g.interp;
    a.epart = g.epart;
    a.n_eblk = g.n_eblk;
    a.ty_a = g.ty_a;
    a.ty_c = g.ty_c;
    a.yz_kxb = g.yz_kxb;
    a.err = c->d_err;
    a.climb_img = g.climb_img;
    a.hdir = (const T*)g.hdir;
    a.llg_a = T(1.0 / (1.0 + c->alpha * c->alpha));
    a.llg_b = T(c->alpha / (1.0 + c->alpha * c->alpha));
    return a;
}

// Rows per CTA and block sizes of the x-forward (a) and x-inverse (c) kernels and the shared memory
// they need.
void set_rows(Group& g, int ty_a, int ty_c, int thr_a = 256, int thr_c = 256) {
    const size_t cs = 2 * (size_t)g.rbytes;
    if (g.dipole && f128_x(g.rbytes, g.Px)) {
        ty_a = f128_x_rows(ty_a);
        ty_c = f128_x_rows(ty_c);
    }
    const bool x2 = g.dipole && x2p_ok(g.rbytes, g.Px);  // two-pass x kernels: fixed rows per CTA
    if (x2) ty_a = ty_c = kX2Rows;
    g.ty_a = ty_a;
    g.ty_c = ty_c;
    g.thr_a = thr_a;
    g.thr_c = thr_c;
    g.smem_a = (size_t)(g.Px + 3 * g.ty_a * g.lsx) * cs;
    g.smem_c = (size_t)(g.Px + 3 * g.ty_c * g.lsx) * cs + 32 * 2 * kEvalTerms * sizeof(double);
    if (g.dipole && f128_x(g.rbytes, g.Px)) {  // the launchers derive these shapes themselves
        g.thr_a = f128_x_threads(ty_a);
        g.thr_c = f128_x_threads(ty_c);
        g.smem_a = f128_x_smem(ty_a);
        g.smem_c = f128_x_smem(ty_c);
    }
    if (x2) {
        g.thr_a = g.thr_c = kX2Threads;
        g.smem_a = x2_smem(g.Px, false);
        g.smem_c = x2_smem(g.Px, true);
    }
    g.smem_c_eval = g.smem_c;
    g.n_eblk = g.nz * ((g.ny + g.ty_c - 1) / g.ty_c);
}

// Launch shapes of one size group (shared memory, rows per CTA, block sizes).
void configure_group(Group& g) {
    const size_t cs = 2 * (size_t)g.rbytes;  // complex element
    g.lsx = fft_line_stride(g.Px);
    g.lsy = fft_line_stride(g.Py);
    // x kernels: 256 threads; rows per CTA such that the 3*rows lines take one FFT pass and the
    // shared memory allows several resident CTAs
    // default: the largest row count whose 3*rows lines take one FFT pass of a 512-thread block
    int ty = 1;
    for (int cand : {16, 8, 5, 4, 2}) {
        if (cand <= g.ny && 3 * cand <= fft_lines_per_pass(512, g.Px) &&
            (size_t)(g.Px + 3 * cand * g.lsx) * cs <= 96 * 1024) {
            ty = cand;
            break;
        }
    }
    if (g.dipole && f128_x(g.rbytes, g.Px)) ty = 8;  // 384 threads
    set_rows(g, ty, ty, 512, 512);
    // y/z kernel: all 3*nz lines of one (pair, kx) in shared memory, plus the kx slab of the tensor
    // spectrum when it is small enough to stage
    g.thr_b = kMaxThreadsYz;
    g.smem_b = (size_t)(g.Py + 3 * g.nz * g.lsy) * cs;
    const size_t slab = (size_t)(g.Py / 2 + 1) * g.nz * 6 * (size_t)g.rbytes;
    if (slab <= 24 * 1024) g.smem_b += slab;
    if (g.dipole && f128_yz(g.rbytes, g.Py, g.nz)) {
        bool stage = false;
        g.thr_b = f128_yz_threads(g.nz);
        g.smem_b = f128_yz_smem(g.nz, g.Py, &stage);
    }
    if (g.dipole && yz2p_ok(g.rbytes, g.Py, g.nz, g.Px)) {
        g.thr_b = kYz2Threads;
        g.smem_b = yz2p_smem(g.Py, g.nz, yz2p_kxb_use(g.nz, g.yz_kxb));
    }
}

// The two-pass y/z kernel's shared memory for the group's column count (after the autotuner's choice).
void configure_yz_smem(Group& g) {
    if (g.dipole && yz2p_ok(g.rbytes, g.Py, g.nz, g.Px)) g.smem_b = yz2p_smem(g.Py, g.nz, yz2p_kxb_use(g.nz, g.yz_kxb));
}

template <typename T> ss_status build_tensor_spectrum(ss_ctx* c, Group& g) {
    const int Px = g.Px, Py = g.Py, nz = g.nz;
    const size_t plane = (size_t)Px * Py;
    const size_t n = (size_t)6 * nz * plane;
    std::vector<double2> host(n, make_double2(0.0, 0.0));
    for (int dz = 0; dz < nz; ++dz)
        for (int dy = -(g.ny - 1); dy <= g.ny - 1; ++dy)
            for (int dx = -(g.nx - 1); dx <= g.nx - 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                double d[6];
                dipole_tensor_at(dx, dy, dz, d);
                const int ix = ((dx % Px) + Px) % Px, iy = ((dy % Py) + Py) % Py;
                for (int k = 0; k < 6; ++k) host[((size_t)k * nz + dz) * plane + (size_t)iy * Px + ix].x = d[k];
            }
    double2 *d_data = nullptr, *d_twx = nullptr, *d_twy = nullptr;
    CUDA_TRY(c, cudaMalloc(&d_data, n * sizeof(double2)));
    auto twx = twiddles(Px), twy = twiddles(Py);
    cudaError_t e = cudaMalloc(&d_twx, Px * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&d_twy, Py * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_data, host.data(), n * sizeof(double2), cudaMemcpyHostToDevice, c->cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_twx, twx.data(), Px * sizeof(double2), cudaMemcpyHostToDevice, c->cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_twy, twy.data(), Py * sizeof(double2), cudaMemcpyHostToDevice, c->cs);
    if (e == cudaSuccess) {
        const FftPlan px = make_plan(Px), py = make_plan(Py);
        // x: rows of length Px, contiguous
        launch_fft_strided_f64(d_data, d_twx, px, 6 * nz * Py, 1, 1, 0, Px, c->cs);
        // y: columns of length Py, stride Px
        launch_fft_strided_f64(d_data, d_twy, py, 6 * nz * Px, Px, Px, 1, (long)plane, c->cs);
        launch_extract_octant<T>(d_data, (T*)g.dhat, Px, Py, nz, 4.0 * M_PI / ((double)Px * Py), c->cs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->cs);
    cudaFree(d_data);
    cudaFree(d_twx);
    cudaFree(d_twy);
    if (e != cudaSuccess) return fail(c, SS_ERR_CUDA, "dipole tensor spectrum: %s", cudaGetErrorString(e));
    return SS_OK;
}

template <typename T> ss_status setup_group(ss_ctx* c, Group& g) {
    using C = cplx<T>;
    const size_t M = (size_t)3 * g.N;
    TRY(dalloc(c, &g.s, g.n_img * M * sizeof(T)));
    TRY(dalloc(c, &g.sp, g.n_img * M * sizeof(T)));
    TRY(dalloc(c, (void**)&g.interp, g.n_img * sizeof(InterpEntry)));
    TRY(dalloc(c, &g.prm, g.n_img * sizeof(ImgParam<T>)));
    TRY(dalloc(c, (void**)&g.epart, (size_t)g.n_img * kEvalTerms * g.nz * g.ny * sizeof(double)));  // any rows per CTA
    TRY(dalloc(c, &g.twx, g.Px * sizeof(C)));
    TRY(dalloc(c, &g.twy, g.Py * sizeof(C)));
    TRY(dalloc(c, &g.twxs, g.Px * sizeof(C)));
    TRY(dalloc(c, &g.twys, g.Py * sizeof(C)));
    TRY(dalloc(c, &g.t2x, 2 * g.Px * sizeof(C)));
    TRY(dalloc(c, &g.t2y, 2 * g.Py * sizeof(C)));
    if (g.direct) TRY(dalloc(c, &g.hdir, (size_t)g.n_img * 3 * g.N * sizeof(T)));
    if (g.dipole) {
        TRY(dalloc(c, &g.spec, (size_t)g.n_pairs * g.Px * 3 * g.nz * g.ny * sizeof(C)));
        TRY(dalloc(c, &g.dhat, (size_t)(g.Px / 2 + 1) * (g.Py / 2 + 1) * g.nz * 6 * sizeof(T)));
    }
    // per-image constants
    std::vector<ImgParam<T>> prm(g.n_img);
    const int nstr = (int)g.strs.size();
    int maxK = 0;
    for (int i = 0; i < nstr; ++i) {
        const ss_string_desc& d = c->strs[g.strs[i]].d;
        for (int k = 0; k < d.n_images; ++k) {
            ImgParam<T>& p = prm[g.str_img0[i] + k];
            p.J = T(d.J);
            p.D = T(d.D);
            p.K = T(d.K);
            p.w = (c->opts.dipole == SS_DIPOLE_OFF) ? T(0) : T(d.w);
        }
        maxK = std::max(maxK, d.n_images);
    }
    CUDA_TRY(c, cudaMemcpyAsync(g.prm, prm.data(), prm.size() * sizeof(ImgParam<T>), cudaMemcpyHostToDevice, c->cs));
    auto twx = twiddles(g.Px), twy = twiddles(g.Py);
    std::vector<C> tx(g.Px), ty(g.Py);
    for (int i = 0; i < g.Px; ++i) tx[i] = C{T(twx[i].x), T(twx[i].y)};
    for (int i = 0; i < g.Py; ++i) ty[i] = C{T(twy[i].x), T(twy[i].y)};
    CUDA_TRY(c, cudaMemcpyAsync(g.twx, tx.data(), g.Px * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.twy, ty.data(), g.Py * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    std::vector<C> sx(g.Px, C{T(0), T(0)}), sy(g.Py, C{T(0), T(0)});
    fft_stage_twiddles(g.planx, twx.data(), sx.data());
    fft_stage_twiddles(g.plany, twy.data(), sy.data());
    CUDA_TRY(c, cudaMemcpyAsync(g.twxs, sx.data(), g.Px * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.twys, sy.data(), g.Py * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    std::vector<C> t2x(2 * g.Px), t2y(2 * g.Py);
    two_pass_twiddles(g.Px, twx, t2x.data());
    two_pass_twiddles(g.Py, twy, t2y.data());
    CUDA_TRY(c, cudaMemcpyAsync(g.t2x, t2x.data(), 2 * g.Px * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.t2y, t2y.data(), 2 * g.Py * sizeof(C), cudaMemcpyHostToDevice, c->cs));
    // arc-length bookkeeping
    ArcArgs& a = g.arc;
    a.n_str = nstr;
    a.maxK = maxK;
    // components per tile CTA: 1024 (4 per thread of a 256-thread CTA), more on large lattices so that a
    // string has at most about 128 tiles -- the finisher sums every tile's partial of every distance
    a.tile_elems = 1024 * std::max(1, std::min(16, (int)(M / (1024 * 128))));
    a.n_tiles = (int)((M + a.tile_elems - 1) / a.tile_elems);
    a.kchunk = std::max(1, std::min(8, maxK - 1));
    a.n_kchunks = std::max(1, (maxK - 1 + a.kchunk - 1) / a.kchunk);
    a.reparam = c->opts.reparam_every != 0;
    TRY(dalloc(c, (void**)&g.d_str_img0, nstr * sizeof(int)));
    TRY(dalloc(c, (void**)&g.d_str_K, nstr * sizeof(int)));
    TRY(dalloc(c, (void**)&g.dpart, (size_t)nstr * maxK * a.n_tiles * sizeof(double)));
    TRY(dalloc(c, (void**)&g.e_last, (size_t)nstr * maxK * sizeof(double)));
    const size_t n_cnt = (size_t)nstr;  // tile CTAs finished per string
    TRY(dalloc(c, (void**)&g.arc_cnt, n_cnt * sizeof(unsigned)));
    CUDA_TRY(c, cudaMemsetAsync(g.arc_cnt, 0, n_cnt * sizeof(unsigned), c->cs));
    TRY(dalloc(c, (void**)&g.eval_terms, (size_t)nstr * maxK * 4 * sizeof(double)));
    TRY(dalloc(c, (void**)&g.eval_E, (size_t)nstr * maxK * sizeof(double)));
    TRY(dalloc(c, (void**)&g.eval_cn, (size_t)nstr * maxK * sizeof(double)));
    TRY(dalloc(c, (void**)&g.pair_on, (size_t)g.n_pairs * sizeof(int)));
    CUDA_TRY(c, cudaMemcpyAsync(g.d_str_img0, g.str_img0.data(), nstr * sizeof(int), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.d_str_K, g.str_K.data(), nstr * sizeof(int), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemsetAsync(g.dpart, 0, (size_t)nstr * maxK * a.n_tiles * sizeof(double), c->cs));
    CUDA_TRY(c, cudaMemsetAsync(g.e_last, 0, (size_t)nstr * maxK * sizeof(double), c->cs));
    CUDA_TRY(c, cudaMemsetAsync(g.s, 0, g.n_img * M * sizeof(T), c->cs));
    CUDA_TRY(c, cudaMemsetAsync(g.sp, 0, g.n_img * M * sizeof(T), c->cs));
    a.str_img0 = g.d_str_img0;
    a.str_K = g.d_str_K;
    a.dpart = g.dpart;
    a.e_last = g.e_last;
    a.cnt = g.arc_cnt;
    launch_interp_identity(g.interp, 0, g.n_img, c->cs);
    CUDA_TRY(c, cudaGetLastError());
    if (g.dipole) TRY(build_tensor_spectrum<T>(c, g));
    return SS_OK;
}

// Autotuner: rows per CTA and block size of the x kernels and kx columns per CTA of the two-pass y/z
// kernel, timed with CUDA events on the context's stream (the kernels are data-independent; the buffers
// hold zeros and are cleared again afterwards).  Choices are cached per (lattice, image pairs, precision,
// device) for the life of the process.
struct TuneKey {
    int nx, ny, nz, prec, dev, dipole, pairs;  // the best shape also depends on how many CTAs a launch has
    bool operator==(const TuneKey& o) const {
        return nx == o.nx && ny == o.ny && nz == o.nz && prec == o.prec && dev == o.dev && dipole == o.dipole &&
               pairs == o.pairs;
    }
};
std::vector<std::pair<TuneKey, std::array<int, 5>>> g_tuned;  // (thr_a, ty_a, thr_c, ty_c, yz_kxb)
std::mutex g_tune_mu;

template <typename T> ss_status tune_group(ss_ctx* c, Group& g) {
    // SS_X_CONFIG="thr_a:ty_a:thr_c:ty_c[:kxb]" pins the x-kernel shapes and, optionally, the two-pass y/z
    // kernel's columns per CTA (e.g. to profile the tuned shapes, or to compare both column counts)
    if (const char* env = getenv("SS_X_CONFIG")) {
        int ta = 0, ya = 0, tc = 0, yc = 0, kxb = 0;
        const bool f128 = g.dipole && f128_x((int)real_size(c), g.Px);  // block size follows the rows
        const int n = sscanf(env, "%d:%d:%d:%d:%d", &ta, &ya, &tc, &yc, &kxb);
        if (n >= 4 && (f128 || ((ta == 256 || ta == 512) && (tc == 256 || tc == 512))) && ya >= 1 && yc >= 1 &&
            ya <= g.ny && yc <= g.ny) {  // the x kernels for Px = 128 take 2, 4 or 8 rows (others become 8)
            g.yz_kxb = n == 5 ? kxb : 0;  // a count the kernel does not take falls back to the default
            set_rows(g, ya, yc, ta, tc);
            configure_yz_smem(g);
            return SS_OK;
        }
    }
    const TuneKey key{g.nx, g.ny, g.nz, c->opts.precision, c->device, g.dipole ? 1 : 0, g.n_pairs};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto& e : g_tuned)
            if (e.first == key) {
                const int* v = e.second.data();
                g.yz_kxb = v[4];
                set_rows(g, v[1], v[3], v[0], v[2]);
                configure_yz_smem(g);
                return SS_OK;
            }
    }
    const size_t cs = 2 * real_size(c);
    std::vector<std::pair<int, int>> cands;  // (threads, rows)
    if (g.dipole && x2p_ok((int)real_size(c), g.Px)) {
        cands.push_back({kX2Threads, kX2Rows});  // one shape: nothing to tune
    } else if (g.dipole && f128_x((int)real_size(c), g.Px)) {
        for (int ty : {2, 4, 8})  // 48 threads per row; row counts that divide 16 keep the passes conflict-free
            cands.push_back({f128_x_threads(ty), ty});
    } else {
        for (int thr : {256, 512})
            for (int ty : {1, 2, 4, 5, 8, 10, 16})
                if (ty <= g.ny && (size_t)(g.Px + 3 * ty * g.lsx) * cs + 4096 <= 96 * 1024 &&
                    fft_lines_per_pass(thr, g.Px) >= 1 && 3 * ty <= 2 * fft_lines_per_pass(thr, g.Px))
                    cands.push_back({thr, ty});
    }
    std::vector<int> kxbs;  // y/z columns per CTA
    if (g.dipole && yz2p_ok((int)real_size(c), g.Py, g.nz, g.Px) && yz2p_kxb_alt(g.nz) > 0 &&
        g.Px % yz2p_kxb_alt(g.nz) == 0)
        kxbs = {yz2p_kxb(g.nz), yz2p_kxb_alt(g.nz)};
    if (cands.size() <= 1 && kxbs.size() <= 1) return SS_OK;
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    const int reps = 6, trials = 3;
    auto time_it = [&](auto&& run, float* out) -> ss_status {
        run();
        float ms_best = 1e30f;
        for (int tr = 0; tr < trials; ++tr) {
            CUDA_TRY(c, cudaEventRecord(e0, c->cs));
            for (int r = 0; r < reps; ++r) run();
            CUDA_TRY(c, cudaEventRecord(e1, c->cs));
            CUDA_TRY(c, cudaEventSynchronize(e1));
            CUDA_TRY(c, cudaGetLastError());
            float ms = 0.f;
            CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
            ms_best = std::min(ms_best, ms);
        }
        *out = ms_best;
        return SS_OK;
    };
    float best[2] = {1e30f, 1e30f};
    std::pair<int, int> pick[2] = {{g.thr_a, g.ty_a}, {g.thr_c, g.ty_c}};
    const T dt = T(c->opts.dt);
    if (cands.size() > 1) {
        for (auto [thr, ty] : cands) {
            set_rows(g, ty, ty, thr, thr);
            GroupArgs<T> a = group_args<T>(c, g);
            for (int which = 0; which < 2; ++which) {
                float ms = 0.f;
                TRY(time_it([&]() {
                    if (which == 0)
                        launch_xfwd<T>(a, g.dipole, g.thr_a, g.smem_a, c->cs);
                    else
                        launch_xinv_step<T>(a, g.dipole, dt, g.thr_c, g.smem_c, c->cs);
                }, &ms));
                if (ms < best[which]) {
                    best[which] = ms;
                    pick[which] = {thr, ty};
                }
            }
        }
        set_rows(g, pick[0].second, pick[1].second, pick[0].first, pick[1].first);
    }
    if (kxbs.size() > 1) {
        float best_b = 1e30f;
        int pick_b = kxbs[0];
        for (int kxb : kxbs) {
            g.yz_kxb = kxb;
            GroupArgs<T> a = group_args<T>(c, g);
            float ms = 0.f;
            TRY(time_it([&]() { launch_yz<T>(a, g.thr_b, g.smem_b, c->cs); }, &ms));
            if (ms < best_b) {
                best_b = ms;
                pick_b = kxb;
            }
        }
        g.yz_kxb = pick_b;
        configure_yz_smem(g);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const size_t M = (size_t)3 * g.N * g.n_img * real_size(c);
    CUDA_TRY(c, cudaMemsetAsync(g.s, 0, M, c->cs));
    CUDA_TRY(c, cudaMemsetAsync(g.sp, 0, M, c->cs));
    if (g.spec)
        CUDA_TRY(c, cudaMemsetAsync(g.spec, 0, (size_t)g.n_pairs * g.Px * 3 * g.nz * g.ny * 2 * real_size(c), c->cs));
    CUDA_TRY(c, cudaStreamSynchronize(c->cs));
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned.push_back({key, {g.thr_a, g.ty_a, g.thr_c, g.ty_c, g.yz_kxb}});
    return SS_OK;
}

// The launches of one Euler iteration of group g in the current mode, as timed entries: xfwd, yz (with a
// dipole term), xinv (step, climbing-image or LLG mode), the two climbing-image kernels as one entry,
// arc, spline apply.  Launches entry which_only; which_only < 0 launches nothing and returns the number
// of entries.
template <typename T> int time_entries(ss_ctx* c, Group& g, int which_only) {
    GroupArgs<T> a = group_args<T>(c, g);
    const T dt = T(c->opts.dt);
    int e = 0;
    auto entry = [&](bool on, auto&& launch) {
        if (!on) return;
        if (which_only == e) launch();
        ++e;
    };
    entry(true, [&] { launch_xfwd<T>(a, g.dipole, g.thr_a, g.smem_a, c->cs); });
    entry(g.dipole, [&] { launch_yz<T>(a, g.thr_b, g.smem_b, c->cs); });
    entry(g.direct, [&] { launch_dipole_direct<T>(a, (T*)g.hdir, c->cs); });
    entry(true, [&] {
        if (c->dynamics == SS_DYN_LLG)
            launch_xinv_step_llg<T>(a, g.dipole, dt, g.thr_c, g.smem_c, c->cs);
        else if (c->climb)
            launch_xinv_step_climb<T>(a, g.dipole, dt, (T*)g.hc, g.thr_c, g.smem_c, c->cs);
        else
            launch_xinv_step<T>(a, g.dipole, dt, g.thr_c, g.smem_c, c->cs);
    });
    entry(c->climb != 0, [&] { launch_climb<T>(a, g.arc, dt, (const T*)g.hc, c->cs); });
    entry(true, [&] { launch_arc<T>(a, g.arc, g.thr_arc, c->cs); });
    entry(c->interp == SS_INTERP_SPLINE, [&] { launch_spline_apply<T>(a, g.arc, g.arc.maxK, c->cs); });
    return e;
}

// ---- adaptive Runge-Kutta evolution (Sec. III, Dormand-Prince 5(4)) -------------------------------------
// The Runge-Kutta kinds: the pair (0 Dormand-Prince, 1 Runge-Kutta-Fehlberg) and the control granularity.
int rk_method(const ss_ctx* c) { return c->integrator == SS_INT_RKF45 || c->integrator == SS_INT_RKF45_IMAGE; }
bool rk_per_image(int kind) { return kind == SS_INT_DOPRI5_IMAGE || kind == SS_INT_RKF45_IMAGE; }

RkString rk_fresh(const ss_ctx* c) {
    RkString r{};
    r.step = c->opts.dt;
    r.hs = c->opts.dt;
    return r;
}

template <typename T> RkArgs<T> rk_args(const ss_ctx* c, const Group& g) {
    RkArgs<T> r{};
    r.y0 = (T*)g.rk_y0;
    r.k = (T*)g.rk_k;
    r.y5 = (T*)g.rk_y5;
    r.errp = g.rk_errp;
    r.n_tiles = g.rk_tiles;
    r.st = g.rk_st;
    r.img_sys = g.rk_img_sys;
    r.sys_img0 = g.rk_sys_img0;
    r.sys_cnt = g.rk_sys_cnt;
    r.n_sys = g.rk_nsys;
    r.active = g.rk_active;
    r.T_int = c->opts.dt;
    r.rtol = c->rtol;
    r.atol = c->atol;
    r.dp = dp_coefficients<T>(rk_method(c));
    return r;
}

// Buffers of the group's Runge-Kutta evolution, allocated on first use; the ODE systems (whole strings,
// or single images when per_image) and fresh controller states are uploaded on every call.
ss_status rk_setup(ss_ctx* c, Group& g, bool per_image) {
    const size_t M = (size_t)3 * g.N, L = M * g.n_img, rs = real_size(c);
    if (!g.rk_y0) {
        g.rk_tiles = (int)((M + 1023) / 1024);
        TRY(dalloc(c, &g.rk_y0, L * rs));
        TRY(dalloc(c, &g.rk_k, 7 * L * rs));
        TRY(dalloc(c, &g.rk_y5, L * rs));
        TRY(dalloc(c, (void**)&g.rk_errp, (size_t)g.n_img * g.rk_tiles * sizeof(double)));
        TRY(dalloc(c, (void**)&g.rk_st, g.n_img * sizeof(RkString)));
        TRY(dalloc(c, (void**)&g.rk_img_sys, g.n_img * sizeof(int)));
        TRY(dalloc(c, (void**)&g.rk_sys_img0, g.n_img * sizeof(int)));
        TRY(dalloc(c, (void**)&g.rk_sys_cnt, g.n_img * sizeof(int)));
        TRY(dalloc(c, (void**)&g.rk_active, sizeof(int)));
        TRY(dalloc(c, (void**)&g.interp_ident, g.n_img * sizeof(InterpEntry)));
        CUDA_TRY(c, cudaMemsetAsync(g.rk_k, 0, 7 * L * rs, c->cs));
        launch_interp_identity(g.interp_ident, 0, g.n_img, c->cs);
    }
    std::vector<int> img_sys(g.n_img), sys_img0, sys_cnt;
    for (size_t i = 0; i < g.strs.size(); ++i) {
        if (per_image) {
            for (int k = 0; k < g.str_K[i]; ++k) {
                img_sys[g.str_img0[i] + k] = (int)sys_img0.size();
                sys_img0.push_back(g.str_img0[i] + k);
                sys_cnt.push_back(1);
            }
        } else {
            for (int k = 0; k < g.str_K[i]; ++k) img_sys[g.str_img0[i] + k] = (int)i;
            sys_img0.push_back(g.str_img0[i]);
            sys_cnt.push_back(g.str_K[i]);
        }
    }
    g.rk_nsys = (int)sys_img0.size();
    std::vector<RkString> st(g.rk_nsys, rk_fresh(c));
    const size_t ni = g.n_img * sizeof(int), ns = g.rk_nsys * sizeof(int);
    CUDA_TRY(c, cudaMemcpyAsync(g.rk_img_sys, img_sys.data(), ni, cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.rk_sys_img0, sys_img0.data(), ns, cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.rk_sys_cnt, sys_cnt.data(), ns, cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaMemcpyAsync(g.rk_st, st.data(), st.size() * sizeof(RkString), cudaMemcpyHostToDevice, c->cs));
    CUDA_TRY(c, cudaGetLastError());
    return SS_OK;
}

// The controller states of string r: one system, or one per image.
int rk_first_sys(const ss_ctx* c, const StringRec& r) {
    return rk_per_image(c->integrator) ? r.img0 : r.local;
}
int rk_sys_count(const ss_ctx* c, const StringRec& r) {
    return rk_per_image(c->integrator) ? r.d.n_images : 1;
}

// One attempt round of size group g (Sec. III) on stream st: for every stage i, Y_i from y0 and the
// earlier stages, then k_i = F(Y_i) through the field pipeline (identity table) and the step kernel in
// force mode; then the fifth-order solution with its scaled error, the step-size control and the commit of
// accepted attempts.  The first round of an interval also sums the energies of the state the interval
// starts from (its stage 0 is that state).
template <typename T> void issue_rk_round(ss_ctx* c, Group& g, bool first, cudaStream_t st) {
    GroupArgs<T> ai = group_args<T>(c, g);
    ai.interp = g.interp_ident;
    RkArgs<T> r = rk_args<T>(c, g);
    const size_t stride = (size_t)3 * g.N * g.n_img;
    for (int s = 0; s < r.dp.stages; ++s) {
        launch_rk_assemble<T>(ai, r, s, st);
        launch_xfwd<T>(ai, g.dipole, g.thr_a, g.smem_a, st);
        if (g.dipole) launch_yz<T>(ai, g.thr_b, g.smem_b, st);
        if (g.direct) launch_dipole_direct<T>(ai, (T*)g.hdir, st);
        launch_xinv_force<T>(ai, g.dipole, r.k + s * stride, first && s == 0, c->dynamics == SS_DYN_LLG, g.thr_c,
                             g.smem_c_eval, st);
    }
    launch_rk_finish<T>(ai, r, st);
    launch_rk_control<T>(ai, r, 0, st);
    launch_rk_commit<T>(ai, r, st);
}

// One iteration of size group g captured on stream st (a stream capturing the graph): the reparametrised
// state becomes y0 and a new interval opens; the first attempt round runs unconditionally, the further
// ones inside a conditional WHILE node whose body ends by setting the condition from the group's active
// flag (some system has not reached the end of its interval), so the rounds need no host round trip.
// Then the arc kernel reparametrises (Eqs. 11-12).  The body is captured on c->rk_body.
template <typename T> cudaError_t capture_rk_group_iteration(ss_ctx* c, Group& g, cudaStream_t st) {
    GroupArgs<T> a = group_args<T>(c, g);
    GroupArgs<T> ai = a;
    ai.interp = g.interp_ident;
    RkArgs<T> r = rk_args<T>(c, g);
    launch_xfwd<T>(a, false, g.thr_a, 0, st);  // s = reparametrised state
    cudaError_t e = cudaMemcpyAsync(r.y0, a.s, (size_t)3 * g.N * g.n_img * sizeof(T), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    launch_rk_control<T>(ai, r, 1, st);
    issue_rk_round<T>(c, g, true, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph)) != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h{};
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    launch_rk_condition(h, r.active, st);
    const cudaGraphNode_t* deps = nullptr;
    size_t n_deps = 0;
    if ((e = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &n_deps)) != cudaSuccess) return e;
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if ((e = cudaGraphAddNode(&node, graph, deps, nullptr, n_deps, &p)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return e;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(c->rk_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return e;
    issue_rk_round<T>(c, g, false, c->rk_body);
    launch_rk_condition(h, r.active, c->rk_body);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(c->rk_body, &body_out)) != cudaSuccess) return e;
    launch_arc<T>(a, g.arc, g.thr_arc, st);
    if (c->interp == SS_INTERP_SPLINE) launch_spline_apply<T>(a, g.arc, g.arc.maxK, st);
    return cudaGetLastError();
}

// The launches of one Runge-Kutta iteration of group g with a single attempt round, as the timing entries
// of ss_time_kernels in launch order: the interval's opening (x-forward of the reparametrised state, copy
// into y0, control in its opening mode), per stage its assembly, x-forward, y/z (FFT dipole term), direct
// dipole sums (SS_DIPOLE_DIRECT) and x-inverse in force mode, then finish, control, commit, arc and the
// spline apply kernel (spline on).  An interval that needs more than one attempt is left unfinished (the
// next ss_step opens a new one).  which_only < 0 launches nothing and returns the number of entries.
template <typename T> int rk_time_entries(ss_ctx* c, Group& g, int which_only) {
    GroupArgs<T> a = group_args<T>(c, g);
    GroupArgs<T> ai = a;
    ai.interp = g.interp_ident;
    RkArgs<T> r = rk_args<T>(c, g);
    const size_t stride = (size_t)3 * g.N * g.n_img;
    int e = 0;
    auto entry = [&](bool on, auto&& launch) {
        if (!on) return;
        if (which_only == e) launch();
        ++e;
    };
    entry(true, [&] {
        launch_xfwd<T>(a, false, g.thr_a, 0, c->cs);
        cudaMemcpyAsync(r.y0, a.s, stride * sizeof(T), cudaMemcpyDeviceToDevice, c->cs);
        launch_rk_control<T>(ai, r, 1, c->cs);
    });
    for (int st = 0; st < r.dp.stages; ++st) {
        entry(true, [&] { launch_rk_assemble<T>(ai, r, st, c->cs); });
        entry(true, [&] { launch_xfwd<T>(ai, g.dipole, g.thr_a, g.smem_a, c->cs); });
        entry(g.dipole, [&] { launch_yz<T>(ai, g.thr_b, g.smem_b, c->cs); });
        entry(g.direct, [&] { launch_dipole_direct<T>(ai, (T*)g.hdir, c->cs); });
        entry(true, [&] {
            launch_xinv_force<T>(ai, g.dipole, r.k + st * stride, st == 0, c->dynamics == SS_DYN_LLG, g.thr_c,
                                 g.smem_c_eval, c->cs);
        });
    }
    entry(true, [&] { launch_rk_finish<T>(ai, r, c->cs); });
    entry(true, [&] { launch_rk_control<T>(ai, r, 0, c->cs); });
    entry(true, [&] { launch_rk_commit<T>(ai, r, c->cs); });
    entry(true, [&] { launch_arc<T>(a, g.arc, g.thr_arc, c->cs); });
    entry(c->interp == SS_INTERP_SPLINE, [&] { launch_spline_apply<T>(a, g.arc, g.arc.maxK, c->cs); });
    return e;
}

template <typename F> ss_status capture_branched(ss_ctx* c, const char* what, F issue, cudaGraphExec_t* out);
constexpr int kRkGraphIters = 8;

// Capture `iters` Runge-Kutta iterations of every size group, one graph branch per group as in
// capture_graph: each group loops over its own attempt rounds, so a group whose systems all finished
// their interval waits for no other group's rejected attempts.
ss_status capture_rk_graph(ss_ctx* c, int iters, cudaGraphExec_t* out) {
    if (!c->rk_body) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->rk_body, cudaStreamNonBlocking));
    return capture_branched(
        c, "Runge-Kutta graph",
        [&](Group& g, cudaStream_t st) {
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < iters && e == cudaSuccess; ++i)
                e = use_fp64(c) ? capture_rk_group_iteration<double>(c, g, st) : capture_rk_group_iteration<float>(c, g, st);
            return e;
        },
        out);
}

// n_iter iterations of the adaptive integrator: per iteration every string integrates over opts.dt with
// as many attempt rounds as its step-size control needs, then reparametrises; replayed from graphs of
// kRkGraphIters and of one iteration.
ss_status rk_iterations(ss_ctx* c, int n_iter) {
    const int G = kRkGraphIters;
    if (n_iter >= G && !c->rk_graphN) TRY(capture_rk_graph(c, G, &c->rk_graphN));
    if (n_iter % G && !c->rk_graph1) TRY(capture_rk_graph(c, 1, &c->rk_graph1));
    for (int i = 0; i < n_iter / G; ++i) CUDA_TRY(c, cudaGraphLaunch(c->rk_graphN, c->cs));
    for (int i = 0; i < n_iter % G; ++i) CUDA_TRY(c, cudaGraphLaunch(c->rk_graph1, c->cs));
    return SS_OK;
}

// Issue one iteration (Sec. III) of size group g on stream st.
template <typename T> void issue_group_iteration(ss_ctx* c, Group& g, cudaStream_t st) {
    const T dt = T(c->opts.dt);
    {
        GroupArgs<T> a = group_args<T>(c, g);
        launch_xfwd<T>(a, g.dipole, g.thr_a, g.smem_a, st);
        if (g.dipole) launch_yz<T>(a, g.thr_b, g.smem_b, st);
        if (g.direct) launch_dipole_direct<T>(a, (T*)g.hdir, st);
        if (c->dynamics == SS_DYN_LLG) {
            launch_xinv_step_llg<T>(a, g.dipole, dt, g.thr_c, g.smem_c, st);
        } else if (c->climb) {
            launch_xinv_step_climb<T>(a, g.dipole, dt, (T*)g.hc, g.thr_c, g.smem_c, st);
            launch_climb<T>(a, g.arc, dt, (const T*)g.hc, st);
        } else {
            launch_xinv_step<T>(a, g.dipole, dt, g.thr_c, g.smem_c, st);
        }
        launch_arc<T>(a, g.arc, g.thr_arc, st);
        if (c->interp == SS_INTERP_SPLINE) launch_spline_apply<T>(a, g.arc, g.arc.maxK, st);
    }
}

// The evaluation pipeline (energies, terms, convolution norms; the field into hout when given).  pair_on
// (device flags per image pair, or null) restricts it to the flagged pairs.
template <typename T> void issue_eval(ss_ctx* c, Group& g, T* hout, cudaStream_t st, const int* pair_on = nullptr) {
    GroupArgs<T> a = group_args<T>(c, g);
    a.pair_on = pair_on;
    launch_xfwd<T>(a, g.dipole, g.thr_a, g.smem_a, st);
    if (g.dipole) launch_yz<T>(a, g.thr_b, g.smem_b, st);
    if (g.direct) launch_dipole_direct<T>(a, (T*)g.hdir, st);
    launch_xinv_eval<T>(a, g.dipole, hout, g.thr_c, g.smem_c_eval, st);
    launch_eval_reduce<T>(a, g.arc, g.eval_terms, g.eval_E, g.eval_cn, st);
}

template <typename T> void issue_materialise(ss_ctx* c, Group& g, cudaStream_t st) {
    GroupArgs<T> a = group_args<T>(c, g);
    launch_xfwd<T>(a, false, g.thr_a, 0, st);
}

cudaStream_t user_stream(const ss_ctx* c) { return (cudaStream_t)c->opts.stream; }

ss_status enter(ss_ctx* c) {
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaEventRecord(c->ev_in, user_stream(c)));
    CUDA_TRY(c, cudaStreamWaitEvent(c->cs, c->ev_in, 0));
    return SS_OK;
}

ss_status leave(ss_ctx* c) {
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaEventRecord(c->ev_out, c->cs));
    CUDA_TRY(c, cudaStreamWaitEvent(user_stream(c), c->ev_out, 0));
    return SS_OK;
}

// Synchronise the internal stream and consume the sticky error word.
ss_status sync_check(ss_ctx* c) {
    CUDA_TRY(c, cudaStreamSynchronize(c->cs));
    int h = 0;
    CUDA_TRY(c, cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CUDA_TRY(c, cudaMemset(c->d_err, 0, sizeof(int)));
        if (h & kErrInvalidSpin) return fail(c, SS_ERR_INVALID_ARG, "input spin with zero norm or non-finite component");
        if (h & kErrStepCollapse)
            return fail(c, SS_ERR_NONFINITE, "Runge-Kutta step size collapsed (more than 100000 attempts in one interval)");
        return fail(c, SS_ERR_NONFINITE, "non-finite energy or arc length on the device");
    }
    return SS_OK;
}

ss_status check_string(ss_ctx* c, int string) {
    if (!c) return SS_ERR_INVALID_ARG;
    if (string < 0 || string >= (int)c->strs.size()) return fail(c, SS_ERR_INVALID_ARG, "string index %d out of range", string);
    return SS_OK;
}

ss_status check_dtype(ss_ctx* c, int dtype) {
    if (dtype != SS_DTYPE_F32 && dtype != SS_DTYPE_F64) return fail(c, SS_ERR_INVALID_ARG, "dtype %d", dtype);
    return SS_OK;
}

size_t dtype_size(int dtype) { return dtype == SS_DTYPE_F64 ? 8 : 4; }

// Copy K images of [K][3][N] SoA data (scaled) into a caller buffer ([K][N][3], dtype, host/device).
ss_status export_soa(ss_ctx* c, const void* src, int K, int N, void* out, int dtype, int on_device, double scale) {
    const size_t bytes = (size_t)K * N * 3 * dtype_size(dtype);
    void* dst = on_device ? out : c->stage;
    if (!on_device && bytes > c->stage_bytes) return fail(c, SS_ERR_INVALID_ARG, "staging buffer too small");
    if (use_fp64(c)) {
        if (dtype == SS_DTYPE_F64)
            launch_soa_to_aos<double, double>((const double*)src, (double*)dst, K, N, scale, c->cs);
        else
            launch_soa_to_aos<double, float>((const double*)src, (float*)dst, K, N, (float)scale, c->cs);
    } else {
        if (dtype == SS_DTYPE_F64)
            launch_soa_to_aos<float, double>((const float*)src, (double*)dst, K, N, scale, c->cs);
        else
            launch_soa_to_aos<float, float>((const float*)src, (float*)dst, K, N, (float)scale, c->cs);
    }
    CUDA_TRY(c, cudaGetLastError());
    if (!on_device) CUDA_TRY(c, cudaMemcpyAsync(out, c->stage, bytes, cudaMemcpyDeviceToHost, c->cs));
    return SS_OK;
}

ss_status ensure_hout(ss_ctx* c, Group& g) {
    if (!g.hout) TRY(dalloc(c, &g.hout, (size_t)g.n_img * 3 * g.N * real_size(c)));
    return SS_OK;
}

ss_status evaluate_group(ss_ctx* c, Group& g, bool want_field) {
    if (want_field) TRY(ensure_hout(c, g));
    if (use_fp64(c))
        issue_eval<double>(c, g, want_field ? (double*)g.hout : nullptr, c->cs);
    else
        issue_eval<float>(c, g, want_field ? (float*)g.hout : nullptr, c->cs);
    CUDA_TRY(c, cudaGetLastError());
    return SS_OK;
}

// The FP64 evaluation copy of every size group of an FP32 context (same lattice, strings, constants and
// dipole spectrum, FP64 buffers and kernels), set up on first use.
ss_status ensure_ev64(ss_ctx* c) {
    if (use_fp64(c) || !c->ev64.empty()) return SS_OK;
    std::vector<Group> ev;
    for (const Group& g : c->groups) {
        Group e;
        e.rbytes = 8;
        e.nx = g.nx;
        e.ny = g.ny;
        e.nz = g.nz;
        e.N = g.N;
        e.Px = g.Px;
        e.Py = g.Py;
        e.n_img = g.n_img;
        e.n_pairs = g.n_pairs;
        e.strs = g.strs;
        e.str_img0 = g.str_img0;
        e.str_K = g.str_K;
        e.dipole = g.dipole;
        e.direct = g.direct;
        e.planx = g.planx;
        e.plany = g.plany;
        configure_group(e);
        if (e.smem_a > 227 * 1024 || e.smem_b > 227 * 1024 || e.smem_c > 227 * 1024)
            return fail(c, SS_ERR_INVALID_ARG, "lattice %d x %d x %d: the FP64 evaluation needs more shared memory than a CTA has",
                        g.nx, g.ny, g.nz);
        ev.push_back(e);
    }
    set_smem_limits<double>(227 * 1024);
    for (Group& e : ev) TRY(setup_group<double>(c, e));
    CUDA_TRY(c, cudaStreamSynchronize(c->cs));
    c->ev64 = std::move(ev);
    return SS_OK;
}

// Energies and energy terms of every image of size group gi, evaluated in FP64 (Eqs. 1, 8): on the FP64
// path by its own evaluation, on the FP32 path by the FP64 pipeline applied to the FP32 state (the
// gathered spins widened to FP64), so that the reported energies carry no FP32 convolution round-off.
// *out points at the group whose eval_E / eval_terms hold the result once the stream reaches them.
// The result is cached until the group's path changes, so the strings of a size group share one evaluation.
ss_status evaluate_energies(ss_ctx* c, int gi, const Group** out) {
    Group& g = c->groups[gi];
    if (use_fp64(c)) {
        if (g.eval_epoch != g.state_epoch) TRY(evaluate_group(c, g, false));
        g.eval_epoch = g.state_epoch;
        *out = &g;
        return SS_OK;
    }
    TRY(ensure_ev64(c));
    Group& e = c->ev64[gi];
    if (g.eval_epoch != g.state_epoch) {
        issue_materialise<float>(c, g, c->cs);
        launch_widen_unit((const float*)g.s, (double*)e.sp, g.n_img, g.N, nullptr, c->cs);
        issue_eval<double>(c, e, nullptr, c->cs);
        CUDA_TRY(c, cudaGetLastError());
        g.eval_epoch = g.state_epoch;
    }
    *out = &e;
    return SS_OK;
}

// FP32 contexts: the FP64 energies of the images that can decide a barrier (Sec. III: max_k E_k - E_0) of
// every string of size group gi, for the group's current state, into *out ([image], NaN for the others).
// The FP32 evaluation gives each image's energy E_k with a round-off bound B_k: its local terms are FP32
// per site and summed in FP32 per thread and warp (bounded below), and the dipole term's FFT round-off
// obeys ||d conv||_2 <= eps ||conv||_2, eps = u (2 log2(Px Py) + 3 nz + 4), so |dE_k| <= w (1/2) eps
// ||conv_k||_2 sqrt(N), plus 1e-9 + 1e-13 |E_k| for the FP64 sums.  An image whose upper bound E_k + B_k lies below the
// largest lower bound max_j (E_j - B_j) of its string cannot be the highest one, so only image 0 and the
// remaining images are evaluated in FP64 -- the pairs holding them, on the FP64 evaluation copy.
ss_status barrier_energies(ss_ctx* c, int gi, const std::vector<double>** out) {
    Group& g = c->groups[gi];
    if (g.bar_epoch == g.state_epoch) {
        *out = &g.bar_E;
        return SS_OK;
    }
    TRY(ensure_ev64(c));
    Group& e = c->ev64[gi];
    const int nstr = (int)g.strs.size(), mk = g.arc.maxK;
    std::vector<double> E(g.n_img, NAN), buf((size_t)nstr * mk), cn((size_t)nstr * mk);
    if (g.eval_epoch == g.state_epoch) {  // every image has its FP64 energy already
        CUDA_TRY(c, cudaMemcpyAsync(buf.data(), e.eval_E, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
        TRY(sync_check(c));
        for (int i = 0; i < nstr; ++i)
            for (int k = 0; k < g.str_K[i]; ++k) E[g.str_img0[i] + k] = buf[(size_t)i * mk + k];
    } else {
        TRY(evaluate_group(c, g, false));  // FP32 energies and convolution norms (and the gathered state in s)
        CUDA_TRY(c, cudaMemcpyAsync(buf.data(), g.eval_E, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
        CUDA_TRY(c, cudaMemcpyAsync(cn.data(), g.eval_cn, cn.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
        TRY(sync_check(c));
        const double eps = std::ldexp(1.0, -24) * (2.0 * std::log2((double)g.Px * g.Py) + 3.0 * g.nz + 4.0);
        std::vector<int> on(g.n_pairs, 0);
        for (int i = 0; i < nstr; ++i) {
            const ss_string_desc& d = c->strs[g.strs[i]].d;
            const double w = g.dipole ? std::fabs(d.w) : 0.0;
            const int K = g.str_K[i], img0 = g.str_img0[i];
            // the local terms: computed per site in FP32 from spins renormalised in FP32 (relative error
            // below 20 u per term), summed per thread over at most m sites in FP32 and over a warp by a
            // five-level FP32 tree, then in FP64; |term_i| <= 3 |J| + 2 |D| + |K| per site
            const double m = std::ceil(2.0 * g.ty_c * g.nx / std::max(1, g.thr_c));
            const double u = std::ldexp(1.0, -24);
            const double local = (25.0 + m) * u * (double)g.N * (3.0 * std::fabs(d.J) + 2.0 * std::fabs(d.D) + std::fabs(d.K));
            auto bound = [&](int k) {
                const size_t q = (size_t)i * mk + k;
                return w * 0.5 * eps * std::sqrt(std::max(cn[q], 0.0)) * std::sqrt((double)g.N) * (1.0 + (25.0 + m) * u) +
                       local + 1e-9 + 1e-13 * std::fabs(buf[q]);
            };
            double lo_max = -INFINITY;
            for (int k = 0; k < K; ++k) lo_max = std::max(lo_max, buf[(size_t)i * mk + k] - bound(k));
            for (int k = 0; k < K; ++k)  // the direct dipole sum has no such bound here: every image then
                if (k == 0 || g.direct || !(buf[(size_t)i * mk + k] + bound(k) < lo_max)) on[(img0 + k) >> 1] = 1;
        }
        CUDA_TRY(c, cudaMemcpyAsync(e.pair_on, on.data(), on.size() * sizeof(int), cudaMemcpyHostToDevice, c->cs));
        launch_widen_unit((const float*)g.s, (double*)e.sp, g.n_img, g.N, e.pair_on, c->cs);
        issue_eval<double>(c, e, nullptr, c->cs, e.pair_on);
        CUDA_TRY(c, cudaGetLastError());
        CUDA_TRY(c, cudaMemcpyAsync(buf.data(), e.eval_E, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
        TRY(sync_check(c));
        for (int i = 0; i < nstr; ++i)
            for (int k = 0; k < g.str_K[i]; ++k)
                if (on[(g.str_img0[i] + k) >> 1]) E[g.str_img0[i] + k] = buf[(size_t)i * mk + k];
    }
    g.bar_E = std::move(E);
    g.bar_epoch = g.state_epoch;
    *out = &g.bar_E;
    return SS_OK;
}

ss_status check_paths(ss_ctx* c, const Group& g) {
    for (int id : g.strs)
        if (!c->strs[id].has_path) return fail(c, SS_ERR_STATE, "string %d has no path (call ss_set_path first)", id);
    return SS_OK;
}

// The streams and events of the graph branches (one stream per size group).  The branches run at equal
// priority: launch priorities that favour the largest group (the critical path of a batch iteration), or
// the smallest, made the uneven study's iteration slower, not faster.
ss_status ensure_branches(ss_ctx* c) {
    const int G = (int)c->groups.size();
    if (G > 1 && c->branch.empty()) {
        c->branch.assign(G, nullptr);
        c->branch_ev.assign(G + 1, nullptr);
        for (auto& st : c->branch) CUDA_TRY(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (auto& ev : c->branch_ev) CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    return SS_OK;
}

// Capture into *out what issue(group, stream) launches for every size group.  With several groups each
// group's chain is its own branch of the graph, forked from and joined back into cs, so the groups'
// kernels overlap on the GPU instead of running one group after another (within a branch the launches
// keep their order and programmatic dependent launch).
template <typename F> ss_status capture_branched(ss_ctx* c, const char* what, F issue, cudaGraphExec_t* out) {
    const int G = (int)c->groups.size();
    TRY(ensure_branches(c));
    cudaGraph_t graph = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (G > 1) {
        e = cudaEventRecord(c->branch_ev[0], c->cs);
        for (int b = 0; b < G && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(c->branch[b], c->branch_ev[0], 0);
    }
    for (int gi = 0; gi < G && e == cudaSuccess; ++gi) e = issue(c->groups[gi], G > 1 ? c->branch[gi] : c->cs);
    if (G > 1) {
        for (int b = 0; b < G && e == cudaSuccess; ++b) {
            e = cudaEventRecord(c->branch_ev[b + 1], c->branch[b]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cs, c->branch_ev[b + 1], 0);
        }
    }
    const cudaError_t e_end = cudaStreamEndCapture(c->cs, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, SS_ERR_CUDA, "%s capture: %s", what, cudaGetErrorString(e));
    }
    if (e_end != cudaSuccess) return fail(c, SS_ERR_CUDA, "%s capture: %s", what, cudaGetErrorString(e_end));
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, SS_ERR_CUDA, "%s instantiate: %s", what, cudaGetErrorString(e));
    return SS_OK;
}

// The captured graphs hold kernel sequences and arguments that the variant setters change.
void drop_graphs(ss_ctx* c) {
    for (cudaGraphExec_t* gp : {&c->graph1, &c->graphN, &c->rk_graph1, &c->rk_graphN}) {
        if (*gp) cudaGraphExecDestroy(*gp);
        *gp = nullptr;
    }
}

// Capture `iters` iterations of every size group (one graph branch per group).
ss_status capture_graph(ss_ctx* c, int iters, cudaGraphExec_t* out) {
    return capture_branched(
        c, "graph",
        [&](Group& g, cudaStream_t st) {
            for (int i = 0; i < iters; ++i) {
                if (use_fp64(c))
                    issue_group_iteration<double>(c, g, st);
                else
                    issue_group_iteration<float>(c, g, st);
            }
            return cudaGetLastError();
        },
        out);
}

ss_status validate_desc(const ss_string_desc& d) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1)
        return fail(nullptr, SS_ERR_INVALID_ARG, "lattice dims must be >= 1 (got %d x %d x %d)", d.nx, d.ny, d.nz);
    if ((long long)d.nx * d.ny * d.nz > (1LL << 26))
        return fail(nullptr, SS_ERR_INVALID_ARG, "lattice of %lld sites is too large", (long long)d.nx * d.ny * d.nz);
    if (d.n_images < 2 || d.n_images > kArcMaxK)
        return fail(nullptr, SS_ERR_INVALID_ARG, "n_images must be in [2, %d] (got %d)", kArcMaxK, d.n_images);
    if (!isfinite(d.J) || !isfinite(d.D) || !isfinite(d.K) || !isfinite(d.w))
        return fail(nullptr, SS_ERR_INVALID_ARG, "constants must be finite");
    if (d.nx > 1024 || d.ny > 1024 || d.nz > 64)
        return fail(nullptr, SS_ERR_INVALID_ARG, "nx, ny must be <= 1024 and nz <= 64");
    return SS_OK;
}

}  // namespace

// ===================================================================================================
// C ABI
extern "C" {

void ss_default_opts(ss_opts* o) {
    if (!o) return;
    o->dt = 0.1;
    o->precision = SS_PREC_FP32;
    o->dipole = SS_DIPOLE_FFT;
    o->reparam_every = 1;
    o->stream = nullptr;
}

ss_status ss_create(int nx, int ny, int nz, double J, double D, double K, double w_dip, int n_images,
                    const ss_opts* opts, ss_ctx** out) {
    ss_string_desc d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.J = J;
    d.D = D;
    d.K = K;
    d.w = w_dip;
    d.n_images = n_images;
    return ss_create_batch(1, &d, opts, out);
}

ss_status ss_create_batch(int n_strings, const ss_string_desc* descs, const ss_opts* opts, ss_ctx** out) {
    if (!out) return fail(nullptr, SS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_strings < 1 || !descs) return fail(nullptr, SS_ERR_INVALID_ARG, "need at least one string");
    ss_opts o;
    ss_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.dt > 0.0) || !isfinite(o.dt)) return fail(nullptr, SS_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (o.precision != SS_PREC_FP32 && o.precision != SS_PREC_FP64)
        return fail(nullptr, SS_ERR_INVALID_ARG, "precision %d", o.precision);
    if (o.dipole != SS_DIPOLE_OFF && o.dipole != SS_DIPOLE_FFT && o.dipole != SS_DIPOLE_DIRECT)
        return fail(nullptr, SS_ERR_INVALID_ARG, "dipole mode %d", o.dipole);
    if (o.reparam_every != 0 && o.reparam_every != 1)
        return fail(nullptr, SS_ERR_INVALID_ARG, "reparam_every must be 0 or 1 (got %d)", o.reparam_every);
    for (int i = 0; i < n_strings; ++i) TRY(validate_desc(descs[i]));

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, SS_ERR_CUDA, "no CUDA device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(nullptr, SS_ERR_CUDA, "cudaGetDeviceProperties failed");
    if (prop.major != 10 || prop.minor != 3)
        return fail(nullptr, SS_ERR_CUDA, "libss is built for sm_103a; device %d is sm_%d%d", dev, prop.major, prop.minor);

    ss_ctx* c = new (std::nothrow) ss_ctx();
    if (!c) return fail(nullptr, SS_ERR_OOM, "host allocation failed");
    c->opts = o;
    c->device = dev;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        c->alloc_fn = g_alloc_fn;
        c->free_fn = g_free_fn;
        c->alloc_user = g_alloc_user;
    }
    auto bail = [&](ss_status st) {
        g_create_error = c->err;
        ss_destroy(c);
        return st;
    };
    if (cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(c, SS_ERR_CUDA, "stream/event creation failed"));
    // group strings by lattice size, in order of first appearance
    for (int i = 0; i < n_strings; ++i) {
        const ss_string_desc& d = descs[i];
        int gi = -1;
        for (int k = 0; k < (int)c->groups.size(); ++k)
            if (c->groups[k].nx == d.nx && c->groups[k].ny == d.ny && c->groups[k].nz == d.nz) gi = k;
        if (gi < 0) {
            Group g;
            g.nx = d.nx;
            g.ny = d.ny;
            g.nz = d.nz;
            g.N = d.nx * d.ny * d.nz;
            c->groups.push_back(g);
            gi = (int)c->groups.size() - 1;
        }
        Group& g = c->groups[gi];
        StringRec r{d, gi, (int)g.strs.size(), g.n_img, false};
        g.strs.push_back(i);
        g.str_img0.push_back(g.n_img);
        g.str_K.push_back(d.n_images);
        g.n_img += d.n_images;
        if (o.dipole == SS_DIPOLE_FFT && d.w != 0.0) g.dipole = true;
        if (o.dipole == SS_DIPOLE_DIRECT && d.w != 0.0) g.direct = true;
        c->strs.push_back(r);
    }
    size_t stage = 0;
    for (Group& g : c->groups) {
        g.n_pairs = (g.n_img + 1) / 2;
        g.Px = g.dipole ? padded_len(g.nx) : 1;
        g.Py = g.dipole ? padded_len(g.ny) : 1;
        g.planx = make_plan(g.Px);
        g.plany = make_plan(g.Py);
        g.rbytes = (int)real_size(c);
        configure_group(g);
        const size_t smem_max = 227 * 1024;
        if (g.smem_a > smem_max || g.smem_b > smem_max || g.smem_c > smem_max)
            return bail(fail(c, SS_ERR_INVALID_ARG, "lattice %d x %d x %d needs more shared memory than a CTA has",
                             g.nx, g.ny, g.nz));
        for (int id : g.strs) stage = std::max(stage, (size_t)c->strs[id].d.n_images * g.N * 3 * sizeof(double));
    }
    if (use_fp64(c))
        set_smem_limits<double>(227 * 1024);
    else
        set_smem_limits<float>(227 * 1024);
    {
        ss_status st = dalloc(c, (void**)&c->d_err, sizeof(int));
        if (st != SS_OK) return bail(st);
        st = dalloc(c, &c->stage, stage);
        if (st != SS_OK) return bail(st);
        c->stage_bytes = stage;
        if (cudaMemsetAsync(c->d_err, 0, sizeof(int), c->cs) != cudaSuccess) return bail(fail(c, SS_ERR_CUDA, "memset"));
    }
    for (Group& g : c->groups) {
        ss_status st = use_fp64(c) ? setup_group<double>(c, g) : setup_group<float>(c, g);
        if (st != SS_OK) return bail(st);
        st = use_fp64(c) ? tune_group<double>(c, g) : tune_group<float>(c, g);
        if (st != SS_OK) return bail(st);
    }
    if (cudaStreamSynchronize(c->cs) != cudaSuccess) return bail(fail(c, SS_ERR_CUDA, "setup failed"));
    *out = c;
    return SS_OK;
}

ss_status ss_set_path(ss_ctx* c, int string, const void* spins, int dtype, int on_device) {
    TRY(check_string(c, string));
    TRY(check_dtype(c, dtype));
    if (!spins) return fail(c, SS_ERR_INVALID_ARG, "spins is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    const int K = r.d.n_images;
    const size_t bytes = (size_t)K * g.N * 3 * dtype_size(dtype);
    ++g.state_epoch;
    TRY(enter(c));
    const void* src = spins;
    if (!on_device) {
        CUDA_TRY(c, cudaMemcpyAsync(c->stage, spins, bytes, cudaMemcpyHostToDevice, c->cs));
        src = c->stage;
    }
    const size_t off = (size_t)r.img0 * 3 * g.N;
    if (use_fp64(c)) {
        double* dst = (double*)g.sp + off;
        if (dtype == SS_DTYPE_F64)
            launch_aos_to_soa<double, double>((const double*)src, dst, K, g.N, c->d_err, c->cs);
        else
            launch_aos_to_soa<double, float>((const float*)src, dst, K, g.N, c->d_err, c->cs);
    } else {
        float* dst = (float*)g.sp + off;
        if (dtype == SS_DTYPE_F64)
            launch_aos_to_soa<float, double>((const double*)src, dst, K, g.N, c->d_err, c->cs);
        else
            launch_aos_to_soa<float, float>((const float*)src, dst, K, g.N, c->d_err, c->cs);
    }
    launch_interp_identity(g.interp, r.img0, K, c->cs);
    if (c->climb) {  // no image climbs before the new path's first energies are known
        const int none = -1;
        CUDA_TRY(c, cudaMemcpyAsync(g.arc.kc + r.local, &none, sizeof none, cudaMemcpyHostToDevice, c->cs));
        CUDA_TRY(c, cudaMemsetAsync(g.climb_img + r.img0, 0, (size_t)K * sizeof(int), c->cs));
    }
    if (c->integrator != SS_INT_EULER) {  // the adaptive integrator restarts from step opts.dt on a new path
        const std::vector<RkString> fresh(rk_sys_count(c, r), rk_fresh(c));
        CUDA_TRY(c, cudaMemcpyAsync(g.rk_st + rk_first_sys(c, r), fresh.data(), fresh.size() * sizeof(RkString),
                                    cudaMemcpyHostToDevice, c->cs));
    }
    CUDA_TRY(c, cudaGetLastError());
    ss_status st = sync_check(c);
    TRY(leave(c));
    if (st != SS_OK) return st;
    r.has_path = true;
    return SS_OK;
}

ss_status ss_set_integrator(ss_ctx* c, int kind, double rtol, double atol) {
    if (!c) return SS_ERR_INVALID_ARG;
    if (kind != SS_INT_EULER && kind != SS_INT_DOPRI5 && kind != SS_INT_DOPRI5_IMAGE && kind != SS_INT_RKF45 &&
        kind != SS_INT_RKF45_IMAGE)
        return fail(c, SS_ERR_INVALID_ARG, "unknown integrator %d", kind);
    if (kind != SS_INT_EULER && !(rtol > 0.0 && atol > 0.0 && std::isfinite(rtol) && std::isfinite(atol)))
        return fail(c, SS_ERR_INVALID_ARG, "rtol and atol must be positive and finite");
    if (kind != SS_INT_EULER && c->climb)
        return fail(c, SS_ERR_STATE, "the climbing image is defined for the Euler step only");
    TRY(enter(c));
    if (kind != SS_INT_EULER) {
        for (Group& g : c->groups) TRY(rk_setup(c, g, rk_per_image(kind)));
        c->rtol = rtol;
        c->atol = atol;
    }
    c->integrator = kind;
    drop_graphs(c);
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_set_reparam(ss_ctx* c, int interp, int climb) {
    if (!c) return SS_ERR_INVALID_ARG;
    if (interp != SS_INTERP_LINEAR && interp != SS_INTERP_SPLINE)
        return fail(c, SS_ERR_INVALID_ARG, "unknown interpolation %d", interp);
    if (climb != 0 && climb != 1) return fail(c, SS_ERR_INVALID_ARG, "climb must be 0 or 1");
    if (climb && c->integrator != SS_INT_EULER)
        return fail(c, SS_ERR_STATE, "the climbing image is defined for the Euler step only");
    if (climb && c->dynamics != SS_DYN_STRING)
        return fail(c, SS_ERR_STATE, "the climbing image belongs to the string method, not to the LLG dynamics");
    if (interp == SS_INTERP_SPLINE)
        for (const StringRec& r : c->strs)
            if (r.d.n_images > kSplineMaxK)
                return fail(c, SS_ERR_INVALID_ARG, "the spline takes strings of at most %d images", kSplineMaxK);
    TRY(enter(c));
    for (Group& g : c->groups) {
        ArcArgs& a = g.arc;
        const size_t M = (size_t)3 * g.N, nstr = g.strs.size(), mk = (size_t)a.maxK;
        if (climb && !g.hc) {
            a.c_tiles = (g.N + kClimbTile - 1) / kClimbTile;
            TRY(dalloc(c, &g.hc, g.n_img * M * real_size(c)));
            TRY(dalloc(c, (void**)&g.climb_img, g.n_img * sizeof(int)));
            TRY(dalloc(c, (void**)&a.kc, nstr * sizeof(int)));
            TRY(dalloc(c, (void**)&a.cpart, nstr * a.c_tiles * 2 * sizeof(double)));
            a.climb_img = g.climb_img;
        }
        if (climb) {  // every string starts without a climbing image
            CUDA_TRY(c, cudaMemsetAsync(a.kc, 0xff, nstr * sizeof(int), c->cs));
            CUDA_TRY(c, cudaMemsetAsync(g.climb_img, 0, g.n_img * sizeof(int), c->cs));
        }
        if (interp == SS_INTERP_SPLINE && !a.W) {
            TRY(dalloc(c, (void**)&a.W, nstr * mk * mk * sizeof(double)));
            TRY(dalloc(c, (void**)&a.P, nstr * mk * mk * sizeof(double)));
            TRY(dalloc(c, (void**)&a.wcopy, nstr * mk * sizeof(int)));
            CUDA_TRY(c, cudaMemsetAsync(a.wcopy, 0xff, nstr * mk * sizeof(int), c->cs));
        }
        a.climb = climb;
        a.spline = interp == SS_INTERP_SPLINE;
        a.p_dim = a.spline ? std::min(a.maxK, kSplineSmemP) : 0;
    }
    c->interp = interp;
    c->climb = climb;
    drop_graphs(c);
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_set_dynamics(ss_ctx* c, int kind, double alpha) {
    if (!c) return SS_ERR_INVALID_ARG;
    if (kind != SS_DYN_STRING && kind != SS_DYN_LLG) return fail(c, SS_ERR_INVALID_ARG, "unknown dynamics %d", kind);
    if (kind == SS_DYN_LLG && !(alpha >= 0.0 && std::isfinite(alpha)))
        return fail(c, SS_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    if (kind == SS_DYN_LLG && c->climb)
        return fail(c, SS_ERR_STATE, "the climbing image belongs to the string method, not to the LLG dynamics");
    c->dynamics = kind;
    c->alpha = kind == SS_DYN_LLG ? alpha : 0.0;
    for (Group& g : c->groups) g.arc.reparam = kind == SS_DYN_STRING && c->opts.reparam_every != 0;
    drop_graphs(c);
    return SS_OK;
}

ss_status ss_climbing_image(ss_ctx* c, int string, int* k) {
    TRY(check_string(c, string));
    if (!k) return fail(c, SS_ERR_INVALID_ARG, "output pointer is NULL");
    *k = -1;
    if (!c->climb) return SS_OK;
    const StringRec& r = c->strs[string];
    const Group& g = c->groups[r.group];
    TRY(enter(c));
    CUDA_TRY(c, cudaMemcpyAsync(k, g.arc.kc + r.local, sizeof(int), cudaMemcpyDeviceToHost, c->cs));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_integrator_state(ss_ctx* c, int string, int image, double* step, long long* accepted,
                              long long* rejected) {
    TRY(check_string(c, string));
    if (!step || !accepted || !rejected) return fail(c, SS_ERR_INVALID_ARG, "output pointer is NULL");
    const StringRec& r = c->strs[string];
    if (image < -1 || image >= r.d.n_images)
        return fail(c, SS_ERR_INVALID_ARG, "image %d out of range [-1, %d)", image, r.d.n_images);
    const Group& g = c->groups[r.group];
    std::vector<RkString> h(1, rk_fresh(c));
    if (c->integrator != SS_INT_EULER) {
        h.resize(rk_sys_count(c, r));
        TRY(enter(c));
        CUDA_TRY(c, cudaMemcpyAsync(h.data(), g.rk_st + rk_first_sys(c, r), h.size() * sizeof(RkString),
                                    cudaMemcpyDeviceToHost, c->cs));
        ss_status st = sync_check(c);
        TRY(leave(c));
        if (st != SS_OK) return st;
        if (image >= 0 && h.size() > 1) h = {h[image]};
    }
    *step = h[0].step;
    *accepted = *rejected = 0;
    for (const RkString& x : h) {
        *step = std::min(*step, x.step);
        *accepted += x.acc;
        *rejected += x.rej;
    }
    return SS_OK;
}

ss_status ss_get_path(ss_ctx* c, int string, void* out, int dtype, int on_device) {
    TRY(check_string(c, string));
    TRY(check_dtype(c, dtype));
    if (!out) return fail(c, SS_ERR_INVALID_ARG, "out is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    TRY(check_paths(c, g));
    TRY(enter(c));
    if (use_fp64(c))
        issue_materialise<double>(c, g, c->cs);
    else
        issue_materialise<float>(c, g, c->cs);
    const char* base = (const char*)g.s + (size_t)r.img0 * 3 * g.N * real_size(c);
    TRY(export_soa(c, base, r.d.n_images, g.N, out, dtype, on_device, 1.0));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_step(ss_ctx* c, int n_iter) {
    if (!c) return SS_ERR_INVALID_ARG;
    if (n_iter < 0) return fail(c, SS_ERR_INVALID_ARG, "n_iter < 0");
    for (const Group& g : c->groups) TRY(check_paths(c, g));
    if (n_iter == 0) return SS_OK;
    for (Group& g : c->groups) ++g.state_epoch;
    TRY(enter(c));
    if (c->integrator != SS_INT_EULER) {
        TRY(rk_iterations(c, n_iter));
        return leave(c);
    }
    const int G = c->graphN_iters;
    if (n_iter >= G && !c->graphN) TRY(capture_graph(c, G, &c->graphN));
    if (n_iter % G && !c->graph1) TRY(capture_graph(c, 1, &c->graph1));
    for (int i = 0; i < n_iter / G; ++i) CUDA_TRY(c, cudaGraphLaunch(c->graphN, c->cs));
    for (int i = 0; i < n_iter % G; ++i) CUDA_TRY(c, cudaGraphLaunch(c->graph1, c->cs));
    return leave(c);
}

ss_status ss_energies(ss_ctx* c, int string, double* out) {
    TRY(check_string(c, string));
    if (!out) return fail(c, SS_ERR_INVALID_ARG, "out is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    TRY(check_paths(c, g));
    TRY(enter(c));
    const Group* ev = nullptr;
    TRY(evaluate_energies(c, r.group, &ev));
    CUDA_TRY(c, cudaMemcpyAsync(out, ev->eval_E + (size_t)r.local * ev->arc.maxK, r.d.n_images * sizeof(double),
                                cudaMemcpyDeviceToHost, c->cs));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_step_energies(ss_ctx* c, int string, double* out) {
    TRY(check_string(c, string));
    if (!out) return fail(c, SS_ERR_INVALID_ARG, "out is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    TRY(enter(c));
    CUDA_TRY(c, cudaMemcpyAsync(out, g.e_last + (size_t)r.local * g.arc.maxK, r.d.n_images * sizeof(double),
                                cudaMemcpyDeviceToHost, c->cs));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_barrier(ss_ctx* c, int string, double* dE, int* k_max) {
    TRY(check_string(c, string));
    const int K = c->strs[string].d.n_images;
    std::vector<double> e(K);
    if (use_fp64(c)) {
        TRY(ss_energies(c, string, e.data()));
    } else {  // FP64 energies of the images that can decide the barrier (see barrier_energies)
        StringRec& r = c->strs[string];
        TRY(check_paths(c, c->groups[r.group]));
        TRY(enter(c));
        const std::vector<double>* be = nullptr;
        TRY(barrier_energies(c, r.group, &be));
        TRY(leave(c));
        for (int k = 0; k < K; ++k) e[k] = (*be)[r.img0 + k];  // NaN: cannot be the highest image
    }
    int kb = 0;
    for (int k = 1; k < K; ++k)
        if (e[k] > e[kb]) kb = k;
    if (dE) *dE = e[kb] - e[0];
    if (k_max) *k_max = kb;
    return SS_OK;
}

ss_status ss_field(ss_ctx* c, int string, void* out, int dtype, int on_device) {
    TRY(check_string(c, string));
    TRY(check_dtype(c, dtype));
    if (!out) return fail(c, SS_ERR_INVALID_ARG, "out is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    TRY(check_paths(c, g));
    TRY(enter(c));
    TRY(evaluate_group(c, g, true));
    const char* base = (const char*)g.hout + (size_t)r.img0 * 3 * g.N * real_size(c);
    TRY(export_soa(c, base, r.d.n_images, g.N, out, dtype, on_device, 1.0));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_grad(ss_ctx* c, int string, int image, void* dE_ds, int dtype, int on_device, double* dE_dJDKw) {
    TRY(check_string(c, string));
    StringRec& r = c->strs[string];
    if (image < 0 || image >= r.d.n_images) return fail(c, SS_ERR_INVALID_ARG, "image %d out of range", image);
    if (dE_ds) TRY(check_dtype(c, dtype));
    Group& g = c->groups[r.group];
    TRY(check_paths(c, g));
    TRY(enter(c));
    if (dE_ds) {  // the field in the path's precision
        TRY(evaluate_group(c, g, true));
        const char* base = (const char*)g.hout + (size_t)(r.img0 + image) * 3 * g.N * real_size(c);
        TRY(export_soa(c, base, 1, g.N, dE_ds, dtype, on_device, -1.0));
    }
    if (dE_dJDKw) {  // the energy terms in FP64
        const Group* ev = nullptr;
        TRY(evaluate_energies(c, r.group, &ev));
        CUDA_TRY(c, cudaMemcpyAsync(dE_dJDKw, ev->eval_terms + ((size_t)r.local * ev->arc.maxK + image) * 4,
                                    4 * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
    }
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_energy_terms(ss_ctx* c, int string, double* out) {
    TRY(check_string(c, string));
    if (!out) return fail(c, SS_ERR_INVALID_ARG, "out is NULL");
    StringRec& r = c->strs[string];
    Group& g = c->groups[r.group];
    TRY(check_paths(c, g));
    TRY(enter(c));
    const Group* ev = nullptr;
    TRY(evaluate_energies(c, r.group, &ev));
    CUDA_TRY(c, cudaMemcpyAsync(out, ev->eval_terms + (size_t)r.local * ev->arc.maxK * 4,
                                (size_t)r.d.n_images * 4 * sizeof(double), cudaMemcpyDeviceToHost, c->cs));
    ss_status st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_time_kernels(ss_ctx* c, int reps, double* ms_out, int max_out, int* n_out) {
    if (!c || reps < 1 || !n_out) return c ? fail(c, SS_ERR_INVALID_ARG, "reps >= 1 and n_out required") : SS_ERR_INVALID_ARG;
    for (const Group& g : c->groups) TRY(check_paths(c, g));
    const bool rk = c->integrator != SS_INT_EULER;
    auto entries = [&](Group& g, int which) {
        if (rk) return use_fp64(c) ? rk_time_entries<double>(c, g, which) : rk_time_entries<float>(c, g, which);
        return use_fp64(c) ? time_entries<double>(c, g, which) : time_entries<float>(c, g, which);
    };
    std::vector<int> per_group;
    int nk = 0;
    for (Group& g : c->groups) ++g.state_epoch;  // the strings advance
    for (Group& g : c->groups) {
        per_group.push_back(entries(g, -2));
        nk += per_group.back();
    }
    *n_out = nk;
    std::vector<cudaEvent_t> ev(2 * nk, nullptr);
    for (auto& e : ev) CUDA_TRY(c, cudaEventCreate(&e));
    std::vector<double> acc(nk, 0.0);
    TRY(enter(c));
    ss_status st = SS_OK;
    for (int r = 0; r <= reps && st == SS_OK; ++r) {
        int k = 0;
        for (size_t gi = 0; gi < c->groups.size(); ++gi) {
            Group& g = c->groups[gi];
            for (int which = 0; which < per_group[gi]; ++which) {
                cudaEventRecord(ev[2 * k], c->cs);
                entries(g, which);
                cudaEventRecord(ev[2 * k + 1], c->cs);
                ++k;
            }
        }
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->cs) != cudaSuccess) {
            st = fail(c, SS_ERR_CUDA, "kernel timing launch failed");
            break;
        }
        if (r == 0) continue;  // untimed iteration
        for (int i = 0; i < nk; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            acc[i] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (st != SS_OK) return st;
    for (int i = 0; i < nk && i < max_out; ++i) ms_out[i] = acc[i] / reps;
    st = sync_check(c);
    TRY(leave(c));
    return st;
}

ss_status ss_launch_config(const ss_ctx* c, int string, int out[8]) {
    if (!c || !out || string < 0 || string >= (int)c->strs.size()) return SS_ERR_INVALID_ARG;
    const Group& g = c->groups[c->strs[string].group];
    const int v[8] = {g.Px, g.Py, g.ty_a, g.ty_c, g.thr_a, g.thr_b, g.thr_c, g.n_eblk};
    for (int i = 0; i < 8; ++i) out[i] = v[i];
    return SS_OK;
}

int ss_num_strings(const ss_ctx* c) { return c ? (int)c->strs.size() : 0; }

ss_status ss_string_info(const ss_ctx* c, int string, ss_string_desc* out) {
    if (!c || !out || string < 0 || string >= (int)c->strs.size()) return SS_ERR_INVALID_ARG;
    *out = c->strs[string].d;
    return SS_OK;
}

ss_status ss_set_allocator(ss_alloc_fn alloc, ss_free_fn free, void* user) {
    if ((alloc == nullptr) != (free == nullptr)) {
        g_create_error = "ss_set_allocator: alloc and free must both be given or both be NULL";
        return SS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc_fn = alloc;
    g_free_fn = free;
    g_alloc_user = alloc ? user : nullptr;
    return SS_OK;
}

int ss_kernels_per_iteration(const ss_ctx* c) {
    if (!c) return 0;
    int n = 0;
    for (const Group& g : c->groups)
        n += (g.dipole || g.direct ? 4 : 3) + (c->climb ? 2 : 0) + (c->interp == SS_INTERP_SPLINE ? 1 : 0);
    return n;
}

const char* ss_last_error(const ss_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void ss_destroy(ss_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->cs) cudaStreamSynchronize(c->cs);
    drop_graphs(c);
    if (c->rk_body) cudaStreamDestroy(c->rk_body);
    for (auto st : c->branch)
        if (st) cudaStreamDestroy(st);
    for (auto ev : c->branch_ev)
        if (ev) cudaEventDestroy(ev);
    for (const auto& a : c->allocs) {
        if (c->free_fn)
            c->free_fn(a.first, a.second, c->device, c->opts.stream, c->alloc_user);
        else
            cudaFree(a.first);
    }
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->cs) cudaStreamDestroy(c->cs);
    delete c;
}

}  // extern "C"
