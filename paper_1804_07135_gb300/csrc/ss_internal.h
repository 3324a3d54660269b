// ss_internal.h -- types shared by the host runtime (ss_api.cu) and the kernels (ss_kernels.cuh).
//
// Data layout in device memory, per size group (strings whose lattices have the same dimensions):
//   s, sp   [image][3][N]            spins before / after the step (SoA planes, x fastest), N = nx*ny*nz
//   spec    [pair][Px][3][nz][ny]    complex spectra of image pairs after the x transform (y fastest);
//                                    the y/z kernel overwrites them in place with the field spectra
//   dhat    [Px/2+1][nz*6][Py/2+1]   one octant of the dipole-tensor spectrum (real coefficients),
//                                    [kxo][|dz|*6 + comp][kyo]
// Two images (2p, 2p+1) share one complex field (real part = image 2p, imaginary part = image 2p+1):
// the dipole kernel is real in real space, so one complex convolution serves both images.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ss {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

constexpr int kMaxStages = 16;
constexpr int kMaxThreadsX = 512;   // largest block of the x-transform kernels (256 or 512, autotuned)
constexpr int kMinBlocksX = 2;      // resident 512-thread blocks per SM they are compiled for (64 registers)
constexpr int kMaxThreadsYz = 384;  // block size of the y/z kernel (3 x 128: one z-convolution row per warp)
constexpr int kMinBlocksYz = 2;
constexpr int kYzKxb1 = 4;          // kx columns per CTA of the y/z kernel for single-layer films
constexpr int kMaxThreads128 = 384;  // length-128 x kernels: at most 8 rows of 48 threads
constexpr int kMinBlocks128 = 3;     // resident 384-thread blocks per SM of the length-128 kernels (56 registers)
constexpr int kArcMaxChunk = 8;     // image differences one arc CTA accumulates
constexpr int kArcMaxK = 1024;      // images per string

// Mixed-radix (2, 3, 4, 8) plan of a length-P complex FFT, stages in Stockham order (powers of two
// first, so the stride Ns of every power-of-two stage and of the first radix-3 stage is a power of two).
// Per stage: q = P/R butterflies per line, ns = product of the earlier radices, tw = P/(ns*R) (twiddle
// index step); ns_mask = ns - 1 when ns is a power of two, else -1.
struct FftPlan {
    int P;
    int nstages;
    int radix[kMaxStages];
    int q[kMaxStages];
    int ns[kMaxStages];
    int tw[kMaxStages];
    int ns_mask[kMaxStages];
};

// Shared-memory position of element i of a line: one padding slot per 16 elements, which spreads the
// strided stores of the early FFT stages over all banks.
__host__ __device__ constexpr int fft_pad(int i) { return i + (i >> 4); }
// Line stride (in elements) for lines of length P: padded length, made odd so that a column read
// across consecutive lines touches distinct banks.
__host__ __device__ constexpr int fft_line_stride(int P) { return (P + (P >> 4) + 1) | 1; }

// Reparametrisation source of one image: normalise((1 - t) sp[src0] + t sp[src1]), or an exact copy
// of sp[src0] when copy != 0.  Image indices are local to the size group.
struct InterpEntry {
    int src0, src1;
    double t;          // FP64 weight (Eq. 12)
    float tf, omtf;    // t and 1 - t rounded once, for the FP32 blend
    int copy;
    int pad;
};

// Constants of the string an image belongs to.
template <typename T> struct ImgParam {
    T J, D, K, w;
};

template <typename T> struct GroupArgs {
    int nx, ny, nz, N;
    int Px, Py;
    int n_img, n_pairs;
    int lsx, lsy;  // shared-memory line strides (complex elements) of the x and y transforms
    T* s;
    T* sp;
    cplx<T>* spec;
    const T* dhat;
    const cplx<T>* twx;   // flat twiddle tables W_P^k (runtime plans)
    const cplx<T>* twy;
    const cplx<T>* twxs;  // per-stage twiddle tables (compile-time plans), P entries each
    const cplx<T>* twys;
    // two-pass transforms (P = 128, 192, 256, 384), 2P entries each, laid out so that the lanes of a warp
    // read consecutive entries: [0, P) pass 1, W_P^{n2 (2m + par)} at (2m + par) * P/16 + n2; [P, 2P) pass A,
    // W_P^{k1 (2m + par2)} at P + (2m + par2) * 16 + k1
    const cplx<T>* t2x;
    const cplx<T>* t2y;
    FftPlan planx, plany;
    const ImgParam<T>* prm;
    const InterpEntry* interp;
    double* epart;  // energy partials, [n_eblk][image] (step) or [n_eblk][image][4] (eval)
    int n_eblk;     // = nz * ceil(ny / ty_c)
    int ty_a, ty_c; // y rows per CTA in the x-forward and x-inverse kernels
    int* err;       // sticky error word (bit 1: invalid input spin, bit 2: non-finite value)
    const int* climb_img;  // [n_img] nonzero for the image that climbs this iteration (climbing mode only)
    T llg_a, llg_b;        // precessional dynamics (Eq. 9): 1 / (1 + alpha^2) and alpha / (1 + alpha^2)
    const T* hdir;         // [image][3][N] direct dipole sums (SS_DIPOLE_DIRECT), or null
    const int* pair_on;    // [n_pairs] evaluate only the pairs flagged here (generic kernels), or null: all
    int yz_kxb;            // kx columns per CTA of the two-pass y/z kernel (autotuned; 0: the default)
};
// Energy partials per image of the evaluation mode: the four terms of Eq. 1 (J, D, K, w with the constant
// set to 1) and the squared norm of the dipole convolution (for the FP32 round-off bound of the w term).
constexpr int kEvalTerms = 5;

// Arc-length / reparametrisation bookkeeping of one size group.
struct ArcArgs {
    int n_str;             // strings in the group
    const int* str_img0;   // [n_str] first group-local image of each string
    const int* str_K;      // [n_str] images per string
    int maxK;
    int n_tiles;           // spatial tiles of the 3N component vector
    int tile_elems;        // components per tile
    int kchunk;            // image differences per CTA along the string
    int n_kchunks;
    double* dpart;         // [n_str][maxK][n_tiles] squared-distance partials
    double* e_last;        // [n_str][maxK] energies of the state before the step
    unsigned* cnt;         // [n_str] tile CTAs finished; zero between launches
    int reparam;           // 0: keep images where they are
    // variants (Sec. III leaves the interpolation open and names the climbing image as a refinement)
    int climb;             // climbing image on: the energy CTAs also take tickets, the finisher picks the next one
    int* kc;               // [n_str] image climbing in the current iteration, or -1
    int* climb_img;        // [n_img] flag per image for the next iteration's x-inverse kernel
    double* cpart;         // [n_str][c_tiles][2] (F.tau, tau.tau) partials of the climbing image
    int c_tiles;           // site tiles of kClimbTile per image
    int spline;            // natural cubic spline: the finisher writes W, the apply kernel moves the images
    double* W;             // [n_str][maxK][maxK] interpolation weights phi_k = sum_q W_kq phi*_q, stored in T
    double* P;             // [n_str][maxK][maxK] scratch: d m_i / d y_q of the spline (in T), column q contiguous
    int* wcopy;            // [n_str][maxK] row k is the identity (image kept as it is)
    int p_dim;             // spline operator columns kept in the finisher's dynamic shared memory (0: none)
};

constexpr int kClimbTile = 256;   // sites per CTA of the climbing-image kernels (one per thread)
constexpr int kSplineMaxK = 256;  // longest string the spline variant accepts
constexpr int kSplineSmemP = 64;  // parts of up to 63 segments keep the spline operator P in shared memory

// Adaptive Runge-Kutta evolution (Sec. III, Dormand-Prince 5(4)): controller state of one ODE system
// (a whole string, or one image under per-image step control).
struct RkString {
    double t;           // reduced time reached within the current interval
    double step;        // step carried between attempts and intervals
    double hs;          // step of the current attempt (step cut to end at the interval's end)
    double err;         // error norm of the last attempt
    long long acc, rej; // accepted and rejected attempts since the path was set
    int done;           // the interval is complete
    int accepted;       // the last attempt was accepted
    int attempts;       // attempts in the current interval
    int pad;
};

// An embedded Runge-Kutta pair in the path's precision: `stages` stage rows a (stage i uses a[i][0..i-1]),
// the weights b of the solution carried forward and the error weights e (difference of the two
// solutions' weights).  method 0: Dormand-Prince 5(4) (Dormand and Prince, 1980; 7 stages, the
// fifth-order solution carried); method 1: Runge-Kutta-Fehlberg 4(5) (Fehlberg, 1969; 6 stages, the
// fourth-order solution carried).
template <typename T> struct DpCoef {
    int stages;
    T a[7][6];
    T b[7];
    T e[7];
};
template <typename T> DpCoef<T> dp_coefficients(int method);

// Device buffers and constants of the Runge-Kutta evolution of one size group.
template <typename T> struct RkArgs {
    T* y0;            // [image][3][N] state at the start of the attempt
    T* k;             // [7][image][3][N] stage forces
    T* y5;            // [image][3][N] fifth-order solution of the attempt
    double* errp;     // [image][tile] squared scaled-error partials
    int n_tiles;      // tiles of 1024 components per image
    RkString* st;     // [n_sys]
    const int* img_sys;   // [n_img] system of each image
    const int* sys_img0;  // [n_sys] first image of each system (its images are consecutive)
    const int* sys_cnt;   // [n_sys] images of each system
    int n_sys;
    int* active;      // any system still inside its interval (written by the controller)
    double T_int, rtol, atol;
    DpCoef<T> dp;
};

enum { kErrInvalidSpin = 1, kErrNonFinite = 2, kErrStepCollapse = 4 };

// Length-128 transforms in two register passes (FP32): the x kernels when Px = 128, the y/z kernel
// when Py = 128 and nz is 4 or 8.  16 threads per line; their launch shapes follow from the rows per
// CTA (x kernels) or from nz (y/z kernel), whatever block size and shared memory the caller passes.
constexpr int kF128Line = 145;  // line stride of their exchange buffers (complex elements, 1 mod 16)
constexpr int kF128Buf = 72;    // line stride of the x kernels' 64-point lines (fft_pad positions, 8 mod 16)
inline bool f128_x(int real_bytes, int Px) { return real_bytes == 4 && Px == 128; }
inline bool f128_yz(int real_bytes, int Py, int nz) { return real_bytes == 4 && Py == 128 && (nz == 4 || nz == 8); }
// rows per CTA of the x kernels: 2, 4 or 8 (compile-time); anything else is taken as 8
inline int f128_x_rows(int ty) { return ty == 2 || ty == 4 ? ty : 8; }
inline int f128_x_threads(int rows) { return 48 * rows; }
inline size_t f128_x_smem(int rows) {
    // line buffer, exchange buffer (lines rounded up to a multiple of 4), reduction scratch
    return (size_t)(3 * rows * kF128Buf + (3 * rows + 3) / 4 * 4 * kF128Line) * 8 + 32 * 2 * kEvalTerms * sizeof(double);
}
inline int f128_yz_threads(int nz) { return 48 * nz; }
// The length-128 y/z kernel reads its tensor slab through L1 rather than staging it in shared memory
// (measured faster: the 16 pairs of one kx would otherwise each copy the same slab, and the smaller
// shared footprint leaves more L1).
inline size_t f128_yz_smem(int nz, int Py, bool* stage_dhat) {
    (void)Py;
    *stage_dhat = false;
    return (size_t)2 * 3 * nz * kF128Line * 8;
}


// Lengths 192, 256 and 384 in two register passes (FP32, ss_fft.cuh): a line is R2 = P/16 rows of 16 at
// row stride kT2Row; the y/z kernel for those Py with 1, 4 or 8 layers (24 lines per CTA: 8, 2 or 1 kx
// columns), the x kernels for those Px with kX2Rows rows per CTA.
constexpr int kT2Row = 17;
__host__ __device__ constexpr int t2_line(int P) { return kT2Row * (P / 16); }
constexpr int kYz2Threads = 384;
// kx columns per CTA: the default (24 lines) and the alternative the autotuner also times (12 lines for
// one or four layers); 0 when nz has no two-pass kernel
inline int yz2p_kxb(int nz) { return nz == 1 ? 8 : nz == 4 ? 2 : nz == 8 ? 1 : 0; }
inline int yz2p_kxb_alt(int nz) { return nz == 1 ? 4 : nz == 4 ? 1 : 0; }
inline bool yz2p_ok(int real_bytes, int Py, int nz, int Px) {
    if (real_bytes != 4 || !(Py == 192 || Py == 256 || Py == 384)) return false;
    const int kxb = yz2p_kxb(nz);
    return kxb > 0 && Px % kxb == 0;
}
// columns per CTA a launch uses: the tuned choice when it is one of the two, else the default
inline int yz2p_kxb_use(int nz, int tuned) { return tuned > 0 && (tuned == yz2p_kxb(nz) || tuned == yz2p_kxb_alt(nz)) ? tuned : yz2p_kxb(nz); }
inline size_t yz2p_smem(int Py, int nz, int kxb) { return (size_t)3 * nz * kxb * t2_line(Py) * 8; }
constexpr int kX2Rows = 4;
constexpr int kX2Threads = 384;
__host__ __device__ constexpr int x2_round(int v) { return v + ((16 / kX2Rows - v % 16) + 16) % 16; }
__host__ __device__ constexpr int x2_lsx(int P) { return x2_round(t2_line(P) - 1); }  // transform lines
__host__ __device__ constexpr int x2_lb(int P) { return x2_round(fft_pad(P / 2 - 1) + 1); }  // x-space lines
inline bool x2p_ok(int real_bytes, int Px) { return real_bytes == 4 && (Px == 192 || Px == 256 || Px == 384); }
inline size_t x2_smem(int P, bool inverse) {
    return (size_t)3 * kX2Rows * (x2_lsx(P) + x2_lb(P)) * 8 + (inverse ? 32 * 2 * kEvalTerms * 8 : 0);
}


// ---- launchers (defined in ss_kernels.cuh, instantiated for float and double) ----
template <typename T> void launch_xfwd(const GroupArgs<T>& g, bool do_fft, int nthr, size_t smem, cudaStream_t st);
template <typename T> void launch_yz(const GroupArgs<T>& g, int nthr, size_t smem, cudaStream_t st);
template <typename T>
void launch_xinv_step(const GroupArgs<T>& g, bool do_fft, T dt, int nthr, size_t smem, cudaStream_t st);
template <typename T>
void launch_xinv_eval(const GroupArgs<T>& g, bool do_fft, T* hout, int nthr, size_t smem, cudaStream_t st);
// Runge-Kutta stage: the force of Eq. 13 (or with llg the right-hand side of Eq. 9) at the state in s
// into kout; energy partials when energies
template <typename T>
void launch_xinv_force(const GroupArgs<T>& g, bool do_fft, T* kout, bool energies, bool llg, int nthr, size_t smem,
                       cudaStream_t st);
template <typename T> void launch_xinv_step_climb(const GroupArgs<T>& g, bool do_fft, T dt, T* hc, int nthr, size_t smem,
                                                  cudaStream_t st);
template <typename T> void launch_xinv_step_llg(const GroupArgs<T>& g, bool do_fft, T dt, int nthr, size_t smem,
                                                cudaStream_t st);
template <typename T> void launch_dipole_direct(const GroupArgs<T>& g, T* hdir, cudaStream_t st);
template <typename T> void launch_climb(const GroupArgs<T>& g, const ArcArgs& a, T dt, const T* hc, cudaStream_t st);
template <typename T> void launch_spline_apply(const GroupArgs<T>& g, const ArcArgs& a, int maxK, cudaStream_t st);
template <typename T> void launch_rk_assemble(const GroupArgs<T>& g, const RkArgs<T>& r, int stage, cudaStream_t st);
template <typename T> void launch_rk_finish(const GroupArgs<T>& g, const RkArgs<T>& r, cudaStream_t st);
template <typename T>
void launch_rk_control(const GroupArgs<T>& g, const RkArgs<T>& r, int begin, cudaStream_t st);
template <typename T> void launch_rk_commit(const GroupArgs<T>& g, const RkArgs<T>& r, cudaStream_t st);
void launch_rk_condition(cudaGraphConditionalHandle h, const int* active, cudaStream_t st);
template <typename T> void launch_arc(const GroupArgs<T>& g, const ArcArgs& a, int nthr, cudaStream_t st);
template <typename T>
void launch_eval_reduce(const GroupArgs<T>& g, const ArcArgs& a, double* terms, double* energies, double* cnorm2,
                        cudaStream_t st);
template <typename T, typename Tin>
void launch_aos_to_soa(const Tin* src, T* dst, int K, int N, int* err, cudaStream_t st);
template <typename T, typename Tout>
void launch_soa_to_aos(const T* src, Tout* dst, int K, int N, Tout scale, cudaStream_t st);
void launch_interp_identity(InterpEntry* tab, int img0, int K, cudaStream_t st);
// the FP32 state [K][3][N] handed to the FP64 energy evaluation: every spin renormalised in FP64
void launch_widen_unit(const float* src, double* dst, int K, int N, const int* pair_on, cudaStream_t st);
// FP64 setup of the dipole-tensor spectrum: x then y transforms of the padded real-space tensor
// (data [6*nz][Py][Px] complex, in place), then the octant extraction into dhat.
void launch_fft_strided_f64(double2* data, const double2* tw, const FftPlan& plan, int n_lines, long elem_stride,
                            int inner_count, long inner_stride, long outer_stride, cudaStream_t st);
template <typename T> void set_smem_limits(int bytes);
template <typename T>
void launch_extract_octant(const double2* spec, T* dhat, int Px, int Py, int nz, double scale, cudaStream_t st);

}  // namespace ss
