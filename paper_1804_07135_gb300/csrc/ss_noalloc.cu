// ss_noalloc.cu -- ss_field_noalloc: the effective field of a batch of images without allocating
// device memory.
//
// Who needs it: callers that must not call cudaMalloc -- code running inside an application that
// owns all device memory through its own pool, or a plugin whose host forbids allocation.  Everything
// the field evaluation needs beyond the caller's input and output (the pair spectra, the dipole-tensor
// spectrum and its FP64 build area, twiddles, the SoA copies of spins and field, bookkeeping) lives in
// one file-scope device array, g_scratch, of kNoAllocScratchBytes.  Every GPU that loads libss
// reserves that array until the process exits.
//
// Host code must not use g_scratch's name as a device address (in host code it names a host-side
// stand-in); the device address comes from cudaGetSymbolAddress, taken once per device with that
// device current, on the first call.  The call synchronises its stream and reads an error word back,
// so it refuses a stream that is being captured (before issuing any work) rather than break the capture.
#include <limits.h>
#include <math.h>

#include <mutex>

#include "ss.h"
#include "ss_fft.cuh"
#include "ss_internal.h"

using namespace ss;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

struct ScratchSlot {
    unsigned char* ptr;
    bool ready;
};
std::mutex g_mu;
ScratchSlot g_slots[kMaxDevices];

// Device address of g_scratch on the current device, looked up once per device.
ss_status scratch_of_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_slots[dev].ready) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return SS_ERR_CUDA;
        if (prop.major != 10 || prop.minor != 3) return SS_ERR_CUDA;
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return SS_ERR_CUDA;
        set_smem_limits<float>(227 * 1024);
        g_slots[dev].ptr = static_cast<unsigned char*>(p);
        g_slots[dev].ready = true;
    }
    *out = g_slots[dev].ptr;
    return SS_OK;
}

// ---- sizes and launch shapes: the padded-length rule of the context path; the x-kernel row count is a
// fixed rule of its own (no autotuning), chosen to keep every CTA's shared memory under 48 KB ----
bool smooth23(int m) {
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}
int pad_len(int n) {  // the context's rule: smallest 2^a 3^b >= 2n - 1, or a power of two <= 1/8 longer
    int m = n > 1 ? 2 * n - 1 : 1;
    while (!smooth23(m)) ++m;
    int p2 = 1;
    while (p2 < 2 * n - 1) p2 <<= 1;
    return 8 * p2 <= 9 * m ? p2 : m;
}
FftPlan plan_of(int P) { return fft_make_plan(P); }
int up32(int v) { return ((v + 31) / 32) * 32; }
size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

__global__ void na_twiddles(double2* tw64, float2* tw32, int P) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)P, &s, &c);
        tw64[k] = make_double2(c, -s);
        tw32[k] = make_float2((float)c, (float)-s);
    }
}

// Eq. 7 at every lattice offset (dx, dy, dz >= 0) of the zero-padded, circularly ordered grid:
// data [6][nz][Py][Px] complex, imaginary parts zero, origin zero.
__global__ void na_tensor_fill(double2* data, int nx, int ny, int nz, int Px, int Py) {
    const size_t plane = (size_t)Px * Py, total = plane * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % Px), iy = (int)((i / Px) % Py), dz = (int)(i / plane);
        const int dx = ix <= nx - 1 ? ix : (ix >= Px - (nx - 1) ? ix - Px : INT_MAX);
        const int dy = iy <= ny - 1 ? iy : (iy >= Py - (ny - 1) ? iy - Py : INT_MAX);
        double d[6] = {0, 0, 0, 0, 0, 0};
        if (dx != INT_MAX && dy != INT_MAX && (dx | dy | dz) != 0) {
            const double x = dx, y = dy, z = dz;
            const double r2 = x * x + y * y + z * z;
            const double r = sqrt(r2);
            const double inv3 = 1.0 / (r2 * r), inv5 = inv3 / r2;
            const double c = 0.25 / M_PI;
            d[0] = c * (3.0 * x * x * inv5 - inv3);
            d[1] = c * (3.0 * y * y * inv5 - inv3);
            d[2] = c * (3.0 * z * z * inv5 - inv3);
            d[3] = c * 3.0 * x * y * inv5;
            d[4] = c * 3.0 * x * z * inv5;
            d[5] = c * 3.0 * y * z * inv5;
        }
        for (int k = 0; k < 6; ++k) data[(size_t)k * total + i] = make_double2(d[k], 0.0);
    }
}

// Per-stage twiddle table of a plan from the flat FP64 table (layout of fft_stage_twiddles).
__global__ void na_stage_twiddles(FftPlan p, const double2* tw64, float2* out) {
    int o = 0;
    for (int s = 0; s < p.nstages; ++s) {
        const int R = p.radix[s], Ns = p.ns[s];
        if (Ns == 1) continue;
        for (int e = threadIdx.x; e < Ns * (R - 1); e += blockDim.x) {
            const int jm = e / (R - 1), r = 1 + e % (R - 1);
            const double2 x = tw64[(jm * r * p.tw[s]) % p.P];
            out[o + e] = make_float2((float)x.x, (float)x.y);
        }
        o += Ns * (R - 1);
    }
}

// Two-pass twiddle tables (layout of GroupArgs::t2x / t2y) from the flat FP64 table; zeros when P is not
// a multiple of 16.
__global__ void na_t2_table(int P, const double2* tw64, float2* out) {
    const int R2 = P / 16;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * P; i += gridDim.x * blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (P % 16 == 0) {
            const int e = i < P ? i / R2 : (i - P) / 16, q = i < P ? i % R2 : (i - P) % 16;
            const double2 x = tw64[(q * e) % P];
            v = make_float2((float)x.x, (float)x.y);
        }
        out[i] = v;
    }
}

__global__ void na_params(ImgParam<float>* prm, int n, float J, float D, float K, float w) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        ImgParam<float> p;
        p.J = J;
        p.D = D;
        p.K = K;
        p.w = w;
        prm[k] = p;
    }
}

}  // namespace

extern "C" ss_status ss_field_noalloc(int nx, int ny, int nz, double J, double D, double K, double w, int n_images,
                                      const float* spins, float* field, void* stream) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > 1024 || ny > 1024 || nz > 64 || n_images < 1 || n_images > kArcMaxK)
        return SS_ERR_INVALID_ARG;
    if (!isfinite(J) || !isfinite(D) || !isfinite(K) || !isfinite(w)) return SS_ERR_INVALID_ARG;
    if (!spins || !field) return SS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // a capturing stream would record this call's work into the caller's graph and fail at the
    // synchronisation below: refuse it before issuing anything
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SS_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return SS_ERR_STATE;
    // both arrays must be device memory of the current device (checked on the host, before any launch)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return SS_ERR_CUDA;
        for (const void* ptr : {(const void*)spins, (const void*)field}) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
                cudaGetLastError();  // clear the query's error
                return SS_ERR_INVALID_ARG;
            }
            if (at.type != cudaMemoryTypeDevice || at.device != dev) return SS_ERR_INVALID_ARG;
        }
    }
    const bool dip = w != 0.0;
    const int N = nx * ny * nz;
    const int Px = dip ? pad_len(nx) : 1, Py = dip ? pad_len(ny) : 1;
    const int lsx = fft_line_stride(Px), lsy = fft_line_stride(Py), pairs = (n_images + 1) / 2;
    // launch shapes, as for a context of FP32 precision
    const int thr = kMaxThreadsX, thr_b = kMaxThreadsYz;
    int ty = 1;
    for (int cand = 16; cand >= 2; cand /= 2) {
        if (cand <= ny && 3 * cand <= fft_lines_per_pass(thr, Px) && (size_t)(Px + 3 * cand * lsx) * sizeof(float2) <= 48 * 1024) {
            ty = cand;
            break;
        }
    }
    if (dip && f128_x(4, Px)) ty = f128_x_rows(ty);  // the length-128 x kernels take 2, 4 or 8 rows
    if (dip && x2p_ok(4, Px)) ty = kX2Rows;          // the lengths-192/256/384 x kernels take kX2Rows
    const size_t smem_a = (size_t)(Px + 3 * ty * lsx) * sizeof(float2);
    const size_t smem_c = smem_a + 32 * 2 * kEvalTerms * sizeof(double);
    size_t smem_b = (size_t)(Py + 3 * nz * lsy) * sizeof(float2);
    const size_t slab = (size_t)(Py / 2 + 1) * nz * 6 * sizeof(float);
    if (slab <= 24 * 1024) smem_b += slab;
    if (smem_c > 227 * 1024 || smem_b > 227 * 1024) return SS_ERR_INVALID_ARG;
    const int n_eblk = nz * ((ny + ty - 1) / ty);
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(bytes);
        return o;
    };
    const size_t o_err = take(sizeof(int));
    const size_t o_tw64x = take(Px * sizeof(double2)), o_tw64y = take(Py * sizeof(double2));
    const size_t o_twx = take(Px * sizeof(float2)), o_twy = take(Py * sizeof(float2));
    const size_t o_twxs = take(Px * sizeof(float2)), o_twys = take(Py * sizeof(float2));
    const size_t o_t2x = take(2 * Px * sizeof(float2)), o_t2y = take(2 * Py * sizeof(float2));
    const size_t o_dhat = take(dip ? (size_t)(Px / 2 + 1) * (Py / 2 + 1) * nz * 6 * sizeof(float) : 0);
    const size_t o_prm = take(n_images * sizeof(ImgParam<float>));
    const size_t o_interp = take(n_images * sizeof(InterpEntry));
    const size_t o_epart = take((size_t)n_images * kEvalTerms * n_eblk * sizeof(double));
    const size_t o_work = off;
    const size_t tensor_bytes = dip ? (size_t)6 * nz * Px * Py * sizeof(double2) : 0;
    const size_t o_s = o_work;
    const size_t o_h = o_s + up256((size_t)n_images * 3 * N * sizeof(float));
    const size_t o_spec = o_h + up256((size_t)n_images * 3 * N * sizeof(float));
    const size_t spec_end = o_spec + (dip ? up256((size_t)pairs * Px * 3 * nz * ny * sizeof(float2)) : 0);
    const size_t need = spec_end > o_work + tensor_bytes ? spec_end : o_work + tensor_bytes;
    if (need > kNoAllocScratchBytes) return SS_ERR_INVALID_ARG;  // beyond the built-in scratch
    unsigned char* base = nullptr;
    {
        const ss_status s = scratch_of_current_device(&base);
        if (s != SS_OK) return s;
    }
    int* err = reinterpret_cast<int*>(base + o_err);
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return SS_ERR_CUDA;
    double2* tw64x = reinterpret_cast<double2*>(base + o_tw64x);
    double2* tw64y = reinterpret_cast<double2*>(base + o_tw64y);
    float2* twx = reinterpret_cast<float2*>(base + o_twx);
    float2* twy = reinterpret_cast<float2*>(base + o_twy);
    na_twiddles<<<(Px + 127) / 128, 128, 0, st>>>(tw64x, twx, Px);
    na_twiddles<<<(Py + 127) / 128, 128, 0, st>>>(tw64y, twy, Py);
    float* dhat = reinterpret_cast<float*>(base + o_dhat);
    const FftPlan px = plan_of(Px), py = plan_of(Py);
    float2* twxs = reinterpret_cast<float2*>(base + o_twxs);
    float2* twys = reinterpret_cast<float2*>(base + o_twys);
    na_stage_twiddles<<<1, 256, 0, st>>>(px, tw64x, twxs);
    na_stage_twiddles<<<1, 256, 0, st>>>(py, tw64y, twys);
    float2* t2x = reinterpret_cast<float2*>(base + o_t2x);
    float2* t2y = reinterpret_cast<float2*>(base + o_t2y);
    na_t2_table<<<(2 * Px + 127) / 128, 128, 0, st>>>(Px, tw64x, t2x);
    na_t2_table<<<(2 * Py + 127) / 128, 128, 0, st>>>(Py, tw64y, t2y);
    if (dip) {
        // the tensor spectrum is rebuilt on every call: the build area is shared with the spins below
        double2* tens = reinterpret_cast<double2*>(base + o_work);
        const size_t cells = (size_t)nz * Px * Py;
        na_tensor_fill<<<(int)((cells + 255) / 256 < 4096 ? (cells + 255) / 256 : 4096), 256, 0, st>>>(tens, nx, ny, nz, Px, Py);
        launch_fft_strided_f64(tens, tw64x, px, 6 * nz * Py, 1, 1, 0, Px, st);
        launch_fft_strided_f64(tens, tw64y, py, 6 * nz * Px, Px, Px, 1, (long)Px * Py, st);
        launch_extract_octant<float>(tens, dhat, Px, Py, nz, 4.0 * M_PI / ((double)Px * Py), st);
    }
    ImgParam<float>* prm = reinterpret_cast<ImgParam<float>*>(base + o_prm);
    InterpEntry* interp = reinterpret_cast<InterpEntry*>(base + o_interp);
    na_params<<<(n_images + 127) / 128, 128, 0, st>>>(prm, n_images, (float)J, (float)D, (float)K, (float)w);
    launch_interp_identity(interp, 0, n_images, st);
    float* s = reinterpret_cast<float*>(base + o_s);
    float* h = reinterpret_cast<float*>(base + o_h);
    launch_aos_to_soa<float, float>(spins, s, n_images, N, err, st);
    GroupArgs<float> g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.N = N;
    g.Px = Px;
    g.Py = Py;
    g.n_img = n_images;
    g.n_pairs = pairs;
    g.lsx = lsx;
    g.lsy = lsy;
    g.s = s;
    g.sp = s;  // identity reparametrisation: every image copies itself in place
    g.spec = dip ? reinterpret_cast<float2*>(base + o_spec) : nullptr;
    g.dhat = dhat;
    g.twx = twx;
    g.twy = twy;
    g.twxs = twxs;
    g.twys = twys;
    g.t2x = t2x;
    g.t2y = t2y;
    g.planx = px;
    g.plany = py;
    g.prm = prm;
    g.interp = interp;
    g.epart = reinterpret_cast<double*>(base + o_epart);
    g.n_eblk = n_eblk;
    g.ty_a = ty;
    g.ty_c = ty;
    g.err = err;
    launch_xfwd<float>(g, dip, thr, smem_a, st);
    if (dip) launch_yz<float>(g, thr_b, smem_b, st);
    launch_xinv_eval<float>(g, dip, h, thr, smem_c, st);
    launch_soa_to_aos<float, float>(h, field, n_images, N, 1.0f, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return SS_ERR_CUDA;
    int herr = 0;
    if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SS_ERR_CUDA;
    if (herr & kErrInvalidSpin) return SS_ERR_INVALID_ARG;
    return SS_OK;
}
