// ss_kernels.cuh -- the per-iteration kernels of the string method, templated on the real type
// (float: FP32 spins/fields/FFTs with FP64 reductions; double: the plain FP64 method).
//
// One iteration over a size group is four launches:
//   xfwd   (Sec. III interpolation + Sec. II-A)  materialise s = reparam(sp), x-transform of image pairs
//   yz     (Sec. II-A, Eqs. 6-7)                 y-transform, z-convolution with the tensor spectrum,
//                                                inverse y-transform (in place on the spectra)
//   xinv   (Eqs. 3-5, 8, 10, 13)                 inverse x-transform -> dipole field, local field,
//                                                per-image energy partials, projected step -> sp
//   arc    (Eqs. 11-12)                          squared image distances; the last CTA of each string
//                                                sums energies and distances in a fixed order, scans the
//                                                arc length and writes the interpolation table
#pragma once
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "ss_fft.cuh"

namespace ss {

// ------------------------------------------------------------------------------------------------
// small helpers
template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// FP64 square root and reciprocal from FP32 seeds refined by Newton steps of FP64 multiply-adds only
// (GB300's FP64 division and square root are long instruction sequences); within a few ulp of the
// correctly rounded results for positive finite arguments in FP32 range.
__device__ __forceinline__ double sqrt_nr(double x) {
    if (!(x > 0.0)) return x == 0.0 ? 0.0 : sqrt(x);
    const double y = (double)rsqrtf((float)x);  // ~1e-7 relative
    const double s = x * y;
    const double r = fma(-s, s, x);                // residual x - s^2
    return fma(0.5 * y, r, s);                     // one Newton step: ~1e-14 relative
}
// 1 / sqrt(x) for positive finite x in FP32 range: an FP32 seed and two Newton-Raphson steps for the
// reciprocal square root, y <- y + (y / 2) (1 - x y^2), in FP64 multiply-adds (each step squares the
// relative error: ~1e-7 -> ~1e-14 -> rounding level).
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y = (double)rsqrtf((float)x);
    y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
    y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
    return y;
}
__device__ __forceinline__ double rcp_nr(double x) {
    double r = (double)(1.0f / (float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
}

// Fixed-order block reduction of NV doubles per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_reduce_d(double (&v)[NV], double* scratch /* [32*NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (int w = 0; w < nwarp; ++w) a += scratch[w * NV + k];
            v[k] = a;
        }
    }
}

// Block reduction of NV values per thread: summed in T within each warp (fixed shuffle tree), then
// in FP64 across warps by thread 0 (fixed order).  out valid in thread 0.
template <int NV, typename T>
__device__ __forceinline__ void block_reduce_t2d(T (&v)[NV], double (&out)[NV], double* scratch /* [32*NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp * NV + k] = double(v[k]);
    __syncthreads();
    // warp totals combined in FP64 by a fixed shuffle tree in warp 0 (dependent FP64 operations are
    // slow on GB300, so a log-depth tree instead of a sequential loop)
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = lane < nwarp ? scratch[lane * NV + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            out[k] = a;
        }
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialisation may start
// while its predecessor finishes; griddep_wait() blocks until the predecessor grid has completed and
// its writes are visible (a no-op when launched normally).  Nothing before the wait may read the
// predecessor's output or write global memory.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ------------------------------------------------------------------------------------------------
// Gather of rows [y0, y0+rows) of layer z for pair p: s[img] = normalise((1-t) sp[src0] + t sp[src1])
// (or a copy), written back to s and, when buf is given, to line c*lrows + yy of buf (stride ls,
// fft_pad positions) as re/im of the pair.
template <typename T>
__device__ __forceinline__ void xfwd_gather(const GroupArgs<T>& g, cplx<T>* buf, int ls, int lrows, int p, int z,
                                            int y0, int rows, int tid, int nthr) {
    using C = cplx<T>;
    const int nx = g.nx, N = g.N;
    const int ia = 2 * p;
    // the pair's two table entries, loaded once (the stores below could alias them for the compiler)
    InterpEntry ent[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (ia + h < g.n_img) ent[h] = g.interp[ia + h];
    if constexpr (std::is_same<T, float>::value) {
        if ((nx & 1) == 0) {
            // two adjacent sites (x even, x + 1) per thread: the spin planes move as float2
            const int hx = nx >> 1;
            for (int it = tid; it < rows * hx; it += nthr) {
                const int yy = it / hx, x = 2 * (it - yy * hx);
                const int site = (z * g.ny + y0 + yy) * nx + x;
                float out[2][2][3];  // [image][site][component]
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int im = ia + h;
#pragma unroll
                    for (int k = 0; k < 2; ++k) out[h][k][0] = out[h][k][1] = out[h][k][2] = 0.f;
                    if (im >= g.n_img) continue;
                    const InterpEntry& e = ent[h];
                    const float* a = g.sp + (size_t)e.src0 * 3 * N + site;
                    float2 u[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) u[c] = *reinterpret_cast<const float2*>(a + (size_t)c * N);
                    if (!e.copy) {
                        const float t = e.tf, omt = e.omtf;
                        const float* b = g.sp + (size_t)e.src1 * 3 * N + site;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float2 v = *reinterpret_cast<const float2*>(b + (size_t)c * N);
                            u[c] = make_float2(omt * u[c].x + t * v.x, omt * u[c].y + t * v.y);
                        }
                        const float r0 = rsqrtf(u[0].x * u[0].x + u[1].x * u[1].x + u[2].x * u[2].x);
                        const float r1 = rsqrtf(u[0].y * u[0].y + u[1].y * u[1].y + u[2].y * u[2].y);
#pragma unroll
                        for (int c = 0; c < 3; ++c) u[c] = make_float2(u[c].x * r0, u[c].y * r1);
                    }
                    float* d = g.s + (size_t)im * 3 * N + site;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        *reinterpret_cast<float2*>(d + (size_t)c * N) = u[c];
                        out[h][0][c] = u[c].x;
                        out[h][1][c] = u[c].y;
                    }
                }
                if (buf) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int k = 0; k < 2; ++k)
                            buf[(c * lrows + yy) * ls + fft_pad(x + k)] = C{out[0][k][c], out[1][k][c]};
                }
            }
            return;
        }
    }
    for (int it = tid; it < rows * nx; it += nthr) {
        const int yy = it / nx, x = it - yy * nx;
        const int site = (z * g.ny + y0 + yy) * nx + x;
        T out[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int im = ia + h;
            out[h][0] = out[h][1] = out[h][2] = T(0);
            if (im < g.n_img) {
                const InterpEntry& e = ent[h];
                const T* a = g.sp + (size_t)e.src0 * 3 * N + site;
                T u0 = a[0], u1 = a[N], u2 = a[2 * N];
                if (!e.copy) {
                    const T t = sizeof(T) == 4 ? T(e.tf) : T(e.t);
                    const T omt = sizeof(T) == 4 ? T(e.omtf) : T(1.0 - e.t);
                    const T* b = g.sp + (size_t)e.src1 * 3 * N + site;
                    u0 = omt * u0 + t * b[0];
                    u1 = omt * u1 + t * b[N];
                    u2 = omt * u2 + t * b[2 * N];
                    const T r = rsqrt_t<T>(u0 * u0 + u1 * u1 + u2 * u2);
                    u0 *= r;
                    u1 *= r;
                    u2 *= r;
                }
                T* d = g.s + (size_t)im * 3 * N + site;
                d[0] = u0;
                d[N] = u1;
                d[2 * N] = u2;
                out[h][0] = u0;
                out[h][1] = u1;
                out[h][2] = u2;
            }
        }
        if (buf) {
#pragma unroll
            for (int c = 0; c < 3; ++c) buf[(c * lrows + yy) * ls + fft_pad(x)] = C{out[0][c], out[1][c]};
        }
    }
}

// xfwd: grid (ceil(ny/ty_a), nz, n_pairs).  Each CTA takes rows [y0, y0+rows) of layer z for the two
// images of pair p: s[img] = normalise((1-t) sp[src0] + t sp[src1]) (or a copy), written back to s,
// packed as re/im of 3*rows complex lines, zero-padded to Px and transformed along x.
// Output spec[p][kx][c][z][y].
template <typename T, bool DO_FFT, int PX>
__global__ void __launch_bounds__(kMaxThreadsX, kMinBlocksX) xfwd_kernel(GroupArgs<T> g) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + g.Px;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * g.ty_a;
    const int rows = min(g.ty_a, g.ny - y0);
    const int nx = g.nx;
    if (g.pair_on && !g.pair_on[p]) return;  // uniform over the CTA
    if (DO_FFT)
        for (int i = tid; i < g.Px; i += nthr) tw[i] = PX > 0 ? g.twxs[i] : g.twx[i];
    griddep_wait();
    griddep_launch_dependents();
    xfwd_gather(g, DO_FFT ? buf : (C*)nullptr, g.lsx, rows, p, z, y0, rows, tid, nthr);
    if (!DO_FFT) return;
    const int padw = g.Px - nx;
    for (int it = tid; it < 3 * rows * padw; it += nthr) {
        const int line = it / padw, x = nx + (it - line * padw);
        buf[line * g.lsx + fft_pad(x)] = C{T(0), T(0)};
    }
    __syncthreads();
    fft_lines_any<PX, true, false>(buf, tw, g.planx, g.lsx, 3 * rows, tid, nthr);
    // transpose out: each thread writes the rows of one (kx, c), contiguous in y
    const int Px = PX > 0 ? PX : g.Px;
    C* outp = g.spec + (size_t)p * Px * 3 * g.nz * g.ny;
    for (int kc = tid; kc < Px * 3; kc += nthr) {
        const int kx = kc / 3, c = kc - 3 * kx;
        C* o = outp + ((size_t)kc * g.nz + z) * g.ny + y0;
        const C* b = buf + c * rows * g.lsx + fft_pad(kx);
        for (int yy = 0; yy < rows; ++yy) o[yy] = b[yy * g.lsx];
    }
}

// xfwd for Px = 128 (nx <= 64), ROWS (2, 4 or 8) rows per CTA: the same gather, then the x-transform of
// the 3*ROWS lines in two register passes (f128_pass1/2) with 16 roles per line; the second pass writes
// the spectrum straight to global memory, rows fastest across a warp (the rows of one (kx, c) are
// contiguous there).  Rows past ny (last CTA) are skipped.
template <typename T, int ROWS>
__global__ void __launch_bounds__(kMaxThreadsX, kMinBlocksX) xfwd128_kernel(GroupArgs<T> g) {
    using C = cplx<T>;
    static_assert(16 % ROWS == 0, "the pass-2 role permutation needs ROWS | 16");
    constexpr int L = 3 * ROWS, NQ = 16 / ROWS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // L lines of kF128Buf, fft_pad positions
    C* zx = buf + L * kF128Buf;                // exchange buffer
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * ROWS;
    const int rows = min(ROWS, g.ny - y0);
    const int nx = g.nx;
    const C* __restrict__ tw = g.t2x;  // pass-1 twiddles of length 128
    griddep_wait();
    griddep_launch_dependents();
    xfwd_gather(g, buf, kF128Buf, ROWS, p, z, y0, rows, tid, nthr);
    __syncthreads();
    for (int r = tid; r < 16 * ((L + 3) & ~3); r += nthr) {
        int line, n2, par;
        f128_role1(r, line, n2, par);
        if (line >= L || line % ROWS >= rows) continue;
        const C* b = buf + line * kF128Buf;
        C u[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) u[n1] = 8 * n1 + n2 < nx ? b[fft_pad(8 * n1 + n2)] : C{T(0), T(0)};
        f128_pass1<false>(u, u, n2, par, tw, zx + line * kF128Line);
    }
    __syncthreads();
    // pass 2: role (c, j, yy), yy fastest; k1 = a permutation of j that puts a half-warp's 16 reads (rows
    // yy, k1 spaced by ROWS) in distinct banks
    const size_t kstride = (size_t)3 * g.nz * g.ny;  // between consecutive kx
    C* outp = g.spec + (size_t)p * 128 * kstride + (size_t)z * g.ny + y0;
    for (int r = tid; r < 16 * L; r += nthr) {
        const int c = r / (16 * ROWS), rem = r % (16 * ROWS);
        const int j = rem / ROWS, yy = rem % ROWS;
        if (yy >= rows) continue;
        const int k1 = (j % NQ) * ROWS + j / NQ;
        C v[8];
        f128_pass2(v, zx + (c * ROWS + yy) * kF128Line, k1);
        C* o = outp + (size_t)k1 * kstride + (size_t)c * g.nz * g.ny + yy;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) o[(size_t)16 * k2 * kstride] = v[k2];
    }
}

// ------------------------------------------------------------------------------------------------
// Dipole-tensor spectrum lookup: stored octant value with the per-axis parity signs of Eq. 7's
// components (xx, yy, zz, xy: real; xz, yz: imaginary, returned as the coefficient of i).
// Parities (x, y, z): xx/yy/zz even-even-even, xy odd-odd-even, xz odd-even-odd, yz even-odd-odd.

// yz: grid (Px, n_pairs).  Lines (c, z) of length Py: y-transform (rows y >= ny are zero), then for
// each (ky, z) the field spectrum H_a(z) = sum_{z', b} Dhat_ab(kx, ky, z - z') S_b(z'), then the
// inverse y-transform; rows y < ny are written back in place.  The z-convolution stages up to
// kYzItems (ky, z) results per thread in registers, so one shared buffer serves both transforms.
constexpr int kYzItems = 4;

// z-convolution for a compile-time layer count NZ: one thread per (output component a, ky), a uniform
// across a warp (nthr/3 a multiple of 32), both z loops unrolled so |z - z'| and the z-parity sign are
// constants.  Row a of the tensor: a = x: (xx, xy, i xz); a = y: (xy, yy, i yz); a = z: (i xz, i yz, zz).
// dslab holds the coefficient (kyo, |dz|, comp) at dslab[kyo*dk + (|dz|*6 + comp)*dq].
// INPLACE: lines of A (stride lsy, fft_pad positions) are overwritten with the conjugated result;
// otherwise the result goes to the lines of B (same stride, plain positions) and A is only read.
template <int NZ, bool INPLACE = true, typename T, typename C>
__device__ __forceinline__ void zconv_c(const C* A, C* B, int lsy, int Py, int kx, int Px, const T* dslab, int dk,
                                        int dq, int tid, int nthr) {
    const int hx = Px / 2, hy = Py / 2;
    const T sxg = kx > hx ? T(-1) : T(1);
    const int nk = nthr / 3;
    for (int k0 = 0; k0 < Py; k0 += nk) {
        const int a = tid / nk;
        const int ky = k0 + (tid - a * nk);
        const bool act = a < 3 && ky < Py;
        C out[NZ];
        int pky = 0;
        if (act) {
            const int kyo = min(ky, Py - ky);
            const T syg = ky > hy ? T(-1) : T(1);
            const T* d = dslab + (size_t)kyo * dk;
            pky = INPLACE ? fft_pad(ky) : ky;
            // coefficient slots (xx 0, yy 1, zz 2, xy 3, xz 4, yz 5) and x/y parity signs of row a
            const int i0 = a == 0 ? 0 : (a == 1 ? 3 : 4);
            const int i1 = a == 0 ? 3 : (a == 1 ? 1 : 5);
            const int i2 = a == 0 ? 4 : (a == 1 ? 5 : 2);
            const T f0 = a == 0 ? T(1) : (a == 1 ? sxg * syg : sxg);
            const T f1 = a == 0 ? sxg * syg : (a == 1 ? T(1) : syg);
            const T f2 = a == 0 ? sxg : (a == 1 ? syg : T(1));
            T e0[NZ], e1[NZ], e2[NZ];
#pragma unroll
            for (int q = 0; q < NZ; ++q) {
                e0[q] = d[(q * 6 + i0) * dq] * f0;
                e1[q] = d[(q * 6 + i1) * dq] * f1;
                e2[q] = d[(q * 6 + i2) * dq] * f2;
            }
#pragma unroll
            for (int z = 0; z < NZ; ++z) out[z] = C{T(0), T(0)};
            if constexpr (std::is_same<T, float>::value) {
                // paired FP32 form: out += (e, e) * S and (g, g) * (i S) with i S = (-S.y, S.x); the
                // z-parity sign of the odd terms moves onto the operand, -(i S) = (S.y, -S.x)
                if (a < 2) {
#pragma unroll
                    for (int zp = 0; zp < NZ; ++zp) {
                        const float2 sx = A[(0 * NZ + zp) * lsy + pky];
                        const float2 sy = A[(1 * NZ + zp) * lsy + pky];
                        const float2 sz = A[(2 * NZ + zp) * lsy + pky];
                        const float2 isz = make_float2(-sz.y, sz.x), nisz = make_float2(sz.y, -sz.x);
#pragma unroll
                        for (int z = 0; z < NZ; ++z) {
                            const int q = z >= zp ? z - zp : zp - z;
                            out[z] = __ffma2_rn(make_float2(e0[q], e0[q]), sx, out[z]);
                            out[z] = __ffma2_rn(make_float2(e1[q], e1[q]), sy, out[z]);
                            out[z] = __ffma2_rn(make_float2(e2[q], e2[q]), z >= zp ? isz : nisz, out[z]);
                        }
                    }
                } else {
#pragma unroll
                    for (int zp = 0; zp < NZ; ++zp) {
                        const float2 sx = A[(0 * NZ + zp) * lsy + pky];
                        const float2 sy = A[(1 * NZ + zp) * lsy + pky];
                        const float2 sz = A[(2 * NZ + zp) * lsy + pky];
                        const float2 isx = make_float2(-sx.y, sx.x), nisx = make_float2(sx.y, -sx.x);
                        const float2 isy = make_float2(-sy.y, sy.x), nisy = make_float2(sy.y, -sy.x);
#pragma unroll
                        for (int z = 0; z < NZ; ++z) {
                            const int q = z >= zp ? z - zp : zp - z;
                            out[z] = __ffma2_rn(make_float2(e0[q], e0[q]), z >= zp ? isx : nisx, out[z]);
                            out[z] = __ffma2_rn(make_float2(e1[q], e1[q]), z >= zp ? isy : nisy, out[z]);
                            out[z] = __ffma2_rn(make_float2(e2[q], e2[q]), sz, out[z]);
                        }
                    }
                }
            } else if (a < 2) {
#pragma unroll
                for (int zp = 0; zp < NZ; ++zp) {
                    const C sx = A[(0 * NZ + zp) * lsy + pky];
                    const C sy = A[(1 * NZ + zp) * lsy + pky];
                    const C sz = A[(2 * NZ + zp) * lsy + pky];
#pragma unroll
                    for (int z = 0; z < NZ; ++z) {
                        const int q = z >= zp ? z - zp : zp - z;
                        const T g2 = z >= zp ? e2[q] : -e2[q];  // odd in z
                        out[z].x += e0[q] * sx.x + e1[q] * sy.x - g2 * sz.y;
                        out[z].y += e0[q] * sx.y + e1[q] * sy.y + g2 * sz.x;
                    }
                }
            } else {
#pragma unroll
                for (int zp = 0; zp < NZ; ++zp) {
                    const C sx = A[(0 * NZ + zp) * lsy + pky];
                    const C sy = A[(1 * NZ + zp) * lsy + pky];
                    const C sz = A[(2 * NZ + zp) * lsy + pky];
#pragma unroll
                    for (int z = 0; z < NZ; ++z) {
                        const int q = z >= zp ? z - zp : zp - z;
                        const T g0 = z >= zp ? e0[q] : -e0[q];  // odd in z
                        const T g1 = z >= zp ? e1[q] : -e1[q];  // odd in z
                        out[z].x += -g0 * sx.y - g1 * sy.y + e2[q] * sz.x;
                        out[z].y += g0 * sx.x + g1 * sy.x + e2[q] * sz.y;
                    }
                }
            }
        }
        if constexpr (INPLACE) __syncthreads();
        if (act) {
            // conjugated: the inverse transform is the conjugate of the forward transform of the conjugate
#pragma unroll
            for (int z = 0; z < NZ; ++z) B[(a * NZ + z) * lsy + pky] = cconj(out[z]);
        }
        if constexpr (INPLACE) __syncthreads();
    }
}

// z-convolution for any layer count, in passes of whole ky columns (item = ky * nz + z).
template <typename T, typename C>
__device__ __forceinline__ void zconv_any(C* A, int lsy, int Py, int nz, int kx, int Px, const T* dslab, int dk, int dq,
                                          int tid, int nthr) {
    const int hx = Px / 2, hy = Py / 2;
    const T sxg = kx > hx ? T(-1) : T(1);
    const int n_items = Py * nz;
    const int per_pass = max(nz, ((nthr * kYzItems) / nz) * nz);
    for (int base = 0; base < n_items; base += per_pass) {
        const int end = min(n_items, base + per_pass);
        C res[kYzItems][3];
#pragma unroll
        for (int q = 0; q < kYzItems; ++q) {
            const int it = base + tid + q * nthr;
            if (it < end) {
                const int ky = it / nz, z = it - ky * nz;
                const int kyo = min(ky, Py - ky);
                const T syg = ky > hy ? T(-1) : T(1);
                const T sxy = sxg * syg;
                const T* dcol = dslab + (size_t)kyo * dk;
                const int pky = fft_pad(ky);
                C hx_ = {T(0), T(0)}, hy_ = {T(0), T(0)}, hz_ = {T(0), T(0)};
#pragma unroll 2
                for (int zp = 0; zp < nz; ++zp) {
                    const int dz = z - zp;
                    const T szg = dz < 0 ? T(-1) : T(1);
                    const T* d = dcol + (dz < 0 ? -dz : dz) * 6 * dq;
                    const T dxx = d[0], dyy = d[dq], dzz = d[2 * dq];
                    const T dxy = d[3 * dq] * sxy;
                    const T dxz = d[4 * dq] * (sxg * szg);  // coefficient of i
                    const T dyz = d[5 * dq] * (syg * szg);  // coefficient of i
                    const C sx = A[(0 * nz + zp) * lsy + pky];
                    const C sy = A[(1 * nz + zp) * lsy + pky];
                    const C sz = A[(2 * nz + zp) * lsy + pky];
                    // i*c*S = (-c S.y, c S.x)
                    hx_.x += dxx * sx.x + dxy * sy.x - dxz * sz.y;
                    hx_.y += dxx * sx.y + dxy * sy.y + dxz * sz.x;
                    hy_.x += dxy * sx.x + dyy * sy.x - dyz * sz.y;
                    hy_.y += dxy * sx.y + dyy * sy.y + dyz * sz.x;
                    hz_.x += -dxz * sx.y - dyz * sy.y + dzz * sz.x;
                    hz_.y += dxz * sx.x + dyz * sy.x + dzz * sz.y;
                }
                res[q][0] = hx_;
                res[q][1] = hy_;
                res[q][2] = hz_;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kYzItems; ++q) {
            const int it = base + tid + q * nthr;
            if (it < end) {
                const int ky = it / nz, z = it - ky * nz;
                const int pky = fft_pad(ky);
#pragma unroll
                for (int c = 0; c < 3; ++c) A[(c * nz + z) * lsy + pky] = cconj(res[q][c]);
            }
        }
        __syncthreads();
    }
}

// KXB > 1 (single-layer films): KXB consecutive kx columns per CTA (their spectra are contiguous), so
// the short per-column work is amortised over more lines per barrier; the tensor slab is then read
// through L1 (stage_dhat is ignored).
template <typename T, int PY, int NZ, int KXB = 1>
__global__ void __launch_bounds__(kMaxThreadsYz, kMinBlocksYz) yz_kernel(GroupArgs<T> g, int stage_dhat) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* A = tw + g.Py;  // KXB*3*nz lines of stride lsy
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int kx = blockIdx.x * KXB, p = blockIdx.y;
    if (g.pair_on && !g.pair_on[p]) return;  // uniform over the CTA
    const int Py = PY > 0 ? PY : g.Py;
    const int nz = NZ > 0 ? NZ : g.nz;
    const int ny = g.ny, L = 3 * nz * KXB;
    const int hy = Py / 2;
    const int kxo = min(kx, g.Px - kx);
    C* blk = g.spec + ((size_t)p * g.Px + kx) * 3 * nz * ny;
    // this kx's slab of the tensor-spectrum octant, layout [|dz|*6 + comp][kyo] (a warp over
    // consecutive ky reads consecutive words), staged in shared memory when it fits
    const T* dslab = g.dhat + (size_t)kxo * (hy + 1) * nz * 6;
    const int dk = 1, dq = hy + 1;  // strides of kyo and of (|dz|*6 + comp)
    T* dsm = reinterpret_cast<T*>(A + L * g.lsy);
    if (KXB == 1 && stage_dhat) {
        for (int i = tid; i < (hy + 1) * nz * 6; i += nthr) dsm[i] = dslab[i];
        dslab = dsm;
    }
    for (int i = tid; i < Py; i += nthr) tw[i] = PY > 0 ? g.twys[i] : g.twy[i];
    griddep_wait();
    griddep_launch_dependents();
    for (int it = tid; it < L * Py; it += nthr) {
        const int line = it / Py, y = it - line * Py;  // Py is a constant in the specialised variants
        A[line * g.lsy + fft_pad(y)] = (y < ny) ? blk[line * ny + y] : C{T(0), T(0)};
    }
    __syncthreads();
    fft_lines_any<PY, true, false>(A, tw, g.plany, g.lsy, L, tid, nthr);
    if constexpr (KXB == 1) {
        if constexpr (NZ > 0)
            zconv_c<NZ>(A, A, g.lsy, Py, kx, g.Px, dslab, dk, dq, tid, nthr);
        else
            zconv_any(A, g.lsy, Py, nz, kx, g.Px, dslab, dk, dq, tid, nthr);
    } else {
        static_assert(NZ > 0, "several kx per CTA only with a compile-time layer count");
        for (int b = 0; b < KXB; ++b) {
            const int kxb = kx + b, kxob = min(kxb, g.Px - kxb);
            zconv_c<NZ>(A + (size_t)b * 3 * NZ * g.lsy, A + (size_t)b * 3 * NZ * g.lsy, g.lsy, Py, kxb, g.Px,
                        g.dhat + (size_t)kxob * (hy + 1) * NZ * 6, dk, dq, tid, nthr);
        }
    }
    fft_lines_any<PY, false, true>(A, tw, g.plany, g.lsy, L, tid, nthr);
    for (int it = tid; it < L * ny; it += nthr) {
        const int line = it / ny, y = it - line * ny;
        blk[line * ny + y] = cconj(A[line * g.lsy + fft_pad(y)]);
    }
}

// yz for Py = 128 (ny <= 64), NZ layers: the y-transforms in two register passes each way
// (f128_pass1/2, 16 roles per line, 16 * 3 * NZ threads) around the z-convolution.  Two shared
// regions of 3*NZ lines alternate: R1 = forward exchange, then the z-convolution output; R2 = forward
// output (z-convolution input, stride kLz), then the inverse exchange.
constexpr int kLz = 136;  // line stride of the z-convolution input/output ([line][ky], 8 mod 16)
template <typename T, int NZ>
__global__ void __launch_bounds__(kMaxThreadsYz, kMinBlocks128) yz128_kernel(GroupArgs<T> g, int stage_dhat) {
    using C = cplx<T>;
    constexpr int L = 3 * NZ, hy = 64;
    static_assert(L % 4 == 0, "pass-1 roles take lines in groups of four");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* R1 = reinterpret_cast<C*>(smem_raw);
    C* R2 = R1 + L * kF128Line;
    T* dsm = reinterpret_cast<T*>(R2 + L * kF128Line);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int kx = blockIdx.x, p = blockIdx.y;
    const int ny = g.ny;
    const int kxo = min(kx, g.Px - kx);
    C* blk = g.spec + ((size_t)p * g.Px + kx) * L * ny;
    const T* dslab = g.dhat + (size_t)kxo * (hy + 1) * NZ * 6;
    if (stage_dhat) {
        for (int i = tid; i < (hy + 1) * NZ * 6; i += nthr) dsm[i] = dslab[i];
        dslab = dsm;
    }
    const C* __restrict__ tw = g.t2y;  // pass-1 twiddles of length 128
    griddep_wait();
    griddep_launch_dependents();
    for (int r = tid; r < 16 * L; r += nthr) {
        int line, n2, par;
        f128_role1(r, line, n2, par);
        const C* src = blk + (size_t)line * ny + n2;
        C u[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) u[n1] = 8 * n1 + n2 < ny ? src[8 * n1] : C{T(0), T(0)};
        f128_pass1<false>(u, u, n2, par, tw, R1 + line * kF128Line);
    }
    __syncthreads();
    for (int r = tid; r < 16 * L; r += nthr) {
        const int k1 = r & 15, line = r >> 4;
        C v[8];
        f128_pass2(v, R1 + line * kF128Line, k1);
        C* a = R2 + line * kLz + k1;
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) a[16 * k2] = v[k2];
    }
    __syncthreads();
    zconv_c<NZ, false>(R2, R1, kLz, 128, kx, g.Px, dslab, 1, hy + 1, tid, nthr);
    __syncthreads();
    for (int r = tid; r < 16 * L; r += nthr) {
        int line, n2, par;
        f128_role1(r, line, n2, par);
        const C* b = R1 + line * kLz + n2;
        C u[8], hi[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            u[n1] = b[8 * n1];
            hi[n1] = b[8 * n1 + 64];
        }
        f128_pass1<true>(u, hi, n2, par, tw, R2 + line * kF128Line);
    }
    __syncthreads();
    for (int r = tid; r < 16 * L; r += nthr) {
        const int k1 = r & 15, line = r >> 4;
        C v[8];
        f128_pass2(v, R2 + line * kF128Line, k1);
        C* dst = blk + (size_t)line * ny + k1;
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2)
            if (k1 + 16 * k2 < ny) dst[16 * k2] = cconj(v[k2]);
    }
}

// yz for Py = P in {192, 256, 384} (ny <= P/2), FP32, NZ layers, KXB kx columns per CTA: the y-transforms
// in two register passes each way (t2_pass1 / t2_cols / t2_passB, ss_fft.cuh) on lines held in the
// 17-strided row layout, the z-convolution in place between them.  One shared line per (column, component,
// layer): 3 NZ KXB lines of t2_line(P) complex elements, read from the spectrum in pass 1 and written back
// (rows y < ny) in pass B; one shared-memory round trip per pass instead of one per Stockham stage.
// 384 threads; pass 2 and pass A take one warp per line (16 columns x 2 parities).  Three CTAs per SM,
// two at P = 384 (its 78 KB lines; there the kernel keeps 80 registers, which runs a batch of size groups
// faster than three CTAs of 56 registers would, although one group alone runs faster with three).
template <int NZ, int P>
__device__ __forceinline__ void zconv_t2(float2* A, int kx, int Px, const float* dslab, int tid, int nthr) {
    constexpr int LS = t2_line(P), hy = P / 2, dq = P / 2 + 1;
    const float sxg = kx > Px / 2 ? -1.f : 1.f;
    const int nk = nthr / 3;
    // rounds of nk frequencies; a round reads and writes only its own ky, so one barrier (between its
    // reads and its writes) orders it against every other round
    for (int k0 = 0; k0 < P; k0 += nk) {
        const int a = tid / nk;
        const int ky = k0 + (tid - a * nk);
        const bool act = a < 3 && ky < P;
        float2 out[NZ];
        int pky = 0;
        if (act) {
            const int kyo = min(ky, P - ky);
            const float syg = ky > hy ? -1.f : 1.f;
            const float* d = dslab + kyo;
            pky = t2_pos(ky);
            const int i0 = a == 0 ? 0 : (a == 1 ? 3 : 4);
            const int i1 = a == 0 ? 3 : (a == 1 ? 1 : 5);
            const int i2 = a == 0 ? 4 : (a == 1 ? 5 : 2);
            const float f0 = a == 0 ? 1.f : (a == 1 ? sxg * syg : sxg);
            const float f1 = a == 0 ? sxg * syg : (a == 1 ? 1.f : syg);
            const float f2 = a == 0 ? sxg : (a == 1 ? syg : 1.f);
            float e0[NZ], e1[NZ], e2[NZ];
#pragma unroll
            for (int q = 0; q < NZ; ++q) {
                e0[q] = d[(q * 6 + i0) * dq] * f0;
                e1[q] = d[(q * 6 + i1) * dq] * f1;
                e2[q] = d[(q * 6 + i2) * dq] * f2;
            }
#pragma unroll
            for (int z = 0; z < NZ; ++z) out[z] = make_float2(0.f, 0.f);
            // paired FP32 form as in zconv_c: out += (e, e) * S and (g, g) * (i S), i S = (-S.y, S.x)
            if (a < 2) {
#pragma unroll
                for (int zp = 0; zp < NZ; ++zp) {
                    const float2 sx = A[(0 * NZ + zp) * LS + pky];
                    const float2 sy = A[(1 * NZ + zp) * LS + pky];
                    const float2 sz = A[(2 * NZ + zp) * LS + pky];
                    const float2 isz = make_float2(-sz.y, sz.x), nisz = make_float2(sz.y, -sz.x);
#pragma unroll
                    for (int z = 0; z < NZ; ++z) {
                        const int q = z >= zp ? z - zp : zp - z;
                        out[z] = __ffma2_rn(make_float2(e0[q], e0[q]), sx, out[z]);
                        out[z] = __ffma2_rn(make_float2(e1[q], e1[q]), sy, out[z]);
                        out[z] = __ffma2_rn(make_float2(e2[q], e2[q]), z >= zp ? isz : nisz, out[z]);
                    }
                }
            } else {
#pragma unroll
                for (int zp = 0; zp < NZ; ++zp) {
                    const float2 sx = A[(0 * NZ + zp) * LS + pky];
                    const float2 sy = A[(1 * NZ + zp) * LS + pky];
                    const float2 sz = A[(2 * NZ + zp) * LS + pky];
                    const float2 isx = make_float2(-sx.y, sx.x), nisx = make_float2(sx.y, -sx.x);
                    const float2 isy = make_float2(-sy.y, sy.x), nisy = make_float2(sy.y, -sy.x);
#pragma unroll
                    for (int z = 0; z < NZ; ++z) {
                        const int q = z >= zp ? z - zp : zp - z;
                        out[z] = __ffma2_rn(make_float2(e0[q], e0[q]), z >= zp ? isx : nisx, out[z]);
                        out[z] = __ffma2_rn(make_float2(e1[q], e1[q]), z >= zp ? isy : nisy, out[z]);
                        out[z] = __ffma2_rn(make_float2(e2[q], e2[q]), sz, out[z]);
                    }
                }
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int z = 0; z < NZ; ++z) A[(a * NZ + z) * LS + pky] = cconj(out[z]);
        }
    }
}

template <int P, int NZ, int KXB>
__global__ void __launch_bounds__(kYz2Threads, P == 384 ? 2 : 3) yz2p_kernel(GroupArgs<float> g) {
    using C = float2;
    constexpr int R2 = P / 16, LS = t2_line(P), L = 3 * NZ * KXB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int kx = blockIdx.x * KXB, p = blockIdx.y;
    const int ny = g.ny;
    C* blk = g.spec + ((size_t)p * g.Px + kx) * 3 * NZ * ny;  // KXB consecutive columns are contiguous
    const C* __restrict__ tw = g.twy;                         // W_P^k
    const C* __restrict__ t1 = g.t2y;                         // pass 1
    const C* __restrict__ ta = g.t2y + P;                     // pass A
    griddep_wait();
    griddep_launch_dependents();
    // pass 1, role (n2, line, par), n2 fastest: the zero-padded spectrum lines in, rows of Z out
    for (int r = tid; r < 2 * R2 * L; r += nthr) {
        const int n2 = r % R2, q = r / R2, line = q % L, par = q / L;
        const C* src = blk + (size_t)line * ny + n2;
        C u[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) u[j] = R2 * j + n2 < ny ? src[R2 * j] : make_float2(0.f, 0.f);
        t2_pass1<P>(u, n2, par, t1, A + line * LS);
    }
    __syncthreads();
    // pass 2: one warp per line (lanes = 16 columns x 2 parities)
    for (int r = tid; r < 32 * L; r += nthr) t2_cols<P, false>(A + (r >> 5) * LS, r & 15, (r >> 4) & 1, tw, ta);
    __syncthreads();
#pragma unroll 1
    for (int b = 0; b < KXB; ++b) {
        const int kxb = kx + b, kxo = min(kxb, g.Px - kxb);
        zconv_t2<NZ, P>(A + b * 3 * NZ * LS, kxb, g.Px, g.dhat + (size_t)kxo * (P / 2 + 1) * NZ * 6, tid, nthr);
    }
    __syncthreads();
    // pass A (the inverse transform of the conjugated field spectra, in place by columns)
    for (int r = tid; r < 32 * L; r += nthr) t2_cols<P, true>(A + (r >> 5) * LS, r & 15, (r >> 4) & 1, tw, ta);
    __syncthreads();
    // pass B, role (y2, line, par): rows y < ny back to the spectrum, conjugated
    for (int r = tid; r < 2 * R2 * L; r += nthr) {
        const int y2 = r % R2, q = r / R2, line = q % L, par = q / L;
        C v[8];
        t2_passB(v, A + line * LS, y2, par);
        C* dst = blk + (size_t)line * ny;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int y = y2 + R2 * (2 * m + par);
            if (y < ny) dst[y] = cconj(v[m]);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// h at one site (Eqs. 3-6) from its six neighbours (zero outside the lattice) and the dipole
// convolution:
//   h = J sum_nn s_j - D (s_z^{+x} - s_z^{-x}, s_z^{+y} - s_z^{-y}, -s_x^{+x} + s_x^{-x} - s_y^{+y} + s_y^{-y})
//       + 2 K s_z z + w conv
template <typename T>
__device__ __forceinline__ void local_field(const ImgParam<T>& pr, const T* s0, const T* xp, const T* xm, const T* yp,
                                            const T* ym, const T* zp, const T* zm, const T* conv, T* hf) {
#pragma unroll
    for (int c = 0; c < 3; ++c) hf[c] = pr.J * (xp[c] + xm[c] + yp[c] + ym[c] + zp[c] + zm[c]) + pr.w * conv[c];
    hf[0] += -pr.D * (xp[2] - xm[2]);
    hf[1] += -pr.D * (yp[2] - ym[2]);
    hf[2] += -pr.D * (-xp[0] + xm[0] - yp[1] + ym[1]) + T(2) * pr.K * s0[2];
}
// Eqs. 8, 10, 13 at one site: returns -(1/2) h.s; un = normalise(s + dt (h - (s.h) s))
template <typename T>
__device__ __forceinline__ T step_site(const T* s0, const T* hf, T dt, T* un) {
    const T sh = s0[0] * hf[0] + s0[1] * hf[1] + s0[2] * hf[2];
    T u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = s0[c] + dt * (hf[c] - sh * s0[c]);
    const T r = rsqrt_t<T>(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) un[c] = u[c] * r;
    return T(-0.5) * sh;
}

// Step modes (0, 3, 4 of xinv_sites), FP32, even nx: two adjacent sites (x even, x + 1) per thread and
// pass, so the spin planes move as float2 (one load serves both sites' y and z neighbours, and the inner
// x neighbours come from the pair itself).  eacc[h] accumulates the energy terms of image 2p + h.
template <int MODE>
__device__ __forceinline__ void xinv_sites_step2(const GroupArgs<float>& g, float dt, float* hout, const float2* buf,
                                                 int ls, int p, int z, int y0, int rows, int tid, int nthr,
                                                 const int (&climbs)[2], float (&eacc)[2]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N, hx = nx >> 1;
    const int ia = 2 * p;
    const float2 zero = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int it = tid; it < 2 * rows * hx; it += nthr) {
        const int h = it / (rows * hx);
        const int rem = it - h * rows * hx;
        const int yy = rem / hx, x = 2 * (rem - yy * hx);
        const int im = ia + h;
        if (im >= g.n_img) continue;
        const int y = y0 + yy;
        const int site = (z * ny + y) * nx + x;
        const ImgParam<float> pr = g.prm[im];
        const float* __restrict__ sb = g.s + (size_t)im * 3 * N;
        float2 c0[3], xp[3], xm[3], yp[3], ym[3], zp[3], zm[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* q = sb + (size_t)c * N + site;
            const float2 cur = *reinterpret_cast<const float2*>(q);
            const float l = x > 0 ? q[-1] : 0.f, r = x + 2 < nx ? q[2] : 0.f;
            c0[c] = cur;
            xm[c] = make_float2(l, cur.x);
            xp[c] = make_float2(cur.y, r);
            yp[c] = y + 1 < ny ? *reinterpret_cast<const float2*>(q + nx) : zero;
            ym[c] = y > 0 ? *reinterpret_cast<const float2*>(q - nx) : zero;
            zp[c] = z + 1 < nz ? *reinterpret_cast<const float2*>(q + nx * ny) : zero;
            zm[c] = z > 0 ? *reinterpret_cast<const float2*>(q - nx * ny) : zero;
        }
        float un[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float s0[3], a[3], b[3], cc[3], d[3], e[3], f[3], conv[3], hf[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s0[c] = k ? c0[c].y : c0[c].x;
                a[c] = k ? xp[c].y : xp[c].x;
                b[c] = k ? xm[c].y : xm[c].x;
                cc[c] = k ? yp[c].y : yp[c].x;
                d[c] = k ? ym[c].y : ym[c].x;
                e[c] = k ? zp[c].y : zp[c].x;
                f[c] = k ? zm[c].y : zm[c].x;
                const float2 v = buf[(c * rows + yy) * ls + fft_pad(x + k)];
                conv[c] = h == 0 ? v.x : -v.y;  // conjugate of the forward transform of the conjugate
            }
            local_field(pr, s0, a, b, cc, d, e, f, conv, hf);
            if (MODE == 0 || (MODE == 3 && !climbs[h])) {
                eacc[h] += step_site(s0, hf, dt, un[k]);
            } else {
                const float sh = s0[0] * hf[0] + s0[1] * hf[1] + s0[2] * hf[2];
                eacc[h] += -0.5f * sh;
                if (MODE == 3) {  // the climbing image: its force, stepped by the climbing-image kernels
#pragma unroll
                    for (int c = 0; c < 3; ++c) un[k][c] = hf[c] - sh * s0[c];
                } else {  // Eq. 9
                    const float sxh[3] = {s0[1] * hf[2] - s0[2] * hf[1], s0[2] * hf[0] - s0[0] * hf[2],
                                          s0[0] * hf[1] - s0[1] * hf[0]};
                    float u[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) u[c] = s0[c] + dt * (-g.llg_a * sxh[c] + g.llg_b * (hf[c] - sh * s0[c]));
                    const float r = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
                    for (int c = 0; c < 3; ++c) un[k][c] = u[c] * r;
                }
            }
        }
        float* __restrict__ o = (MODE == 3 && climbs[h] ? hout : g.sp) + (size_t)im * 3 * N + site;
#pragma unroll
        for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(o + (size_t)c * N) = make_float2(un[0][c], un[1][c]);
    }
}

// ------------------------------------------------------------------------------------------------
// Per-site work of the x-inverse kernels on rows [y0, y0+rows) of layer z, pair p; buf holds the
// forward transforms of the conjugated field spectra (line c*rows + yy, fft_pad positions) when
// HAS_CONV.  MODE 0: projected Euler step into sp and energy partials.  MODE 1: FP64 energy terms (and
// the field into hout when given).  MODE 3: MODE 0, except that the image flagged in g.climb_img writes
// its force F = h - (s.h) s into hout instead of stepping (the climbing-image kernels step it).
// MODE 2 (a Runge-Kutta stage): the force F = h - (s.h) s of Eq. 13
// into hout, s as stored (not renormalised); energy partials only when dt != 0.  MODES 4 and 5: as 0 and 2
// with the right-hand side of Eq. 9 (precession and damping, prefactors g.llg_a and g.llg_b).
template <typename T, bool HAS_CONV, int MODE>
__device__ __forceinline__ void xinv_sites(const GroupArgs<T>& g, T dt, T* hout, const cplx<T>* buf, int ls,
                                           double* red, int p, int z, int y0, int rows, int tid, int nthr) {
    using C = cplx<T>;
    const int nx = g.nx, ny = g.ny, nz = g.nz, N = g.N;
    const int ia = 2 * p;
    constexpr int NV = MODE == 1 ? 2 * kEvalTerms : 2;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    T eacc[2] = {T(0), T(0)};  // step mode: the thread's few per-site terms, summed in T before FP64
    float facc[MODE == 1 ? NV : 1] = {};  // FP32 evaluation mode: the same for its terms
    bool done = false;
    int climbs[2] = {0, 0};  // MODE 3: which of the pair's images climbs (uniform per image)
    if constexpr (MODE == 3) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (ia + h < g.n_img) climbs[h] = g.climb_img[ia + h];
    }
    if constexpr ((MODE == 0 || MODE == 3 || MODE == 4) && HAS_CONV && std::is_same<T, float>::value) {
        if ((nx & 1) == 0) {  // uniform over the grid
            xinv_sites_step2<MODE>(g, dt, hout, buf, ls, p, z, y0, rows, tid, nthr, climbs, eacc);
            done = true;
        }
    }
    // two sites per thread per pass; restrict-qualified spin planes let the loads of both be issued
    // before either is stored
#pragma unroll 2
    for (int it = done ? 2 * rows * nx : tid; it < 2 * rows * nx; it += nthr) {
        const int h = it / (rows * nx);
        const int rem = it - h * rows * nx;
        const int yy = rem / nx, x = rem - yy * nx;
        const int im = ia + h;
        if (im >= g.n_img) continue;
        const int y = y0 + yy;
        const int site = (z * ny + y) * nx + x;
        const ImgParam<T> pr = g.prm[im];
        const T* __restrict__ sb = g.s + (size_t)im * 3 * N;
        T s0[3], xp[3], xm[3], yp[3], ym[3], zp[3], zm[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T* q = sb + (size_t)c * N + site;
            s0[c] = q[0];
            xp[c] = x + 1 < nx ? q[1] : T(0);
            xm[c] = x > 0 ? q[-1] : T(0);
            yp[c] = y + 1 < ny ? q[nx] : T(0);
            ym[c] = y > 0 ? q[-nx] : T(0);
            zp[c] = z + 1 < nz ? q[nx * ny] : T(0);
            zm[c] = z > 0 ? q[-nx * ny] : T(0);
        }
        T conv[3] = {T(0), T(0), T(0)};
        if (HAS_CONV) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const C v = buf[(c * rows + yy) * ls + fft_pad(x)];
                conv[c] = h == 0 ? v.x : -v.y;  // conjugate of the forward transform of the conjugate
            }
        } else if (g.hdir) {  // direct dipole sums
#pragma unroll
            for (int c = 0; c < 3; ++c) conv[c] = g.hdir[(size_t)im * 3 * N + (size_t)c * N + site];
        }
        T hf[3];
        local_field(pr, s0, xp, xm, yp, ym, zp, zm, conv, hf);
        if (MODE == 0 || (MODE == 3 && !climbs[h])) {
            T un[3];
            eacc[h] += step_site(s0, hf, dt, un);
            T* __restrict__ o = g.sp + (size_t)im * 3 * N + site;
            o[0] = un[0];
            o[N] = un[1];
            o[2 * N] = un[2];
        } else if (MODE == 2 || MODE == 3) {
            const T sh = s0[0] * hf[0] + s0[1] * hf[1] + s0[2] * hf[2];
            eacc[h] += T(-0.5) * sh;
            T* __restrict__ o = hout + (size_t)im * 3 * N + site;
#pragma unroll
            for (int c = 0; c < 3; ++c) o[(size_t)c * N] = hf[c] - sh * s0[c];
        } else if (MODE == 4 || MODE == 5) {
            // Eq. 9: f = -a (s x h) + b (h - (s.h) s)
            const T sh = s0[0] * hf[0] + s0[1] * hf[1] + s0[2] * hf[2];
            eacc[h] += T(-0.5) * sh;
            const T sxh[3] = {s0[1] * hf[2] - s0[2] * hf[1], s0[2] * hf[0] - s0[0] * hf[2], s0[0] * hf[1] - s0[1] * hf[0]};
            T f[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) f[c] = -g.llg_a * sxh[c] + g.llg_b * (hf[c] - sh * s0[c]);
            if (MODE == 4) {
                T u[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) u[c] = s0[c] + dt * f[c];
                const T r = rsqrt_t<T>(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                T* __restrict__ o = g.sp + (size_t)im * 3 * N + site;
#pragma unroll
                for (int c = 0; c < 3; ++c) o[(size_t)c * N] = u[c] * r;
            } else {
                T* __restrict__ o = hout + (size_t)im * 3 * N + site;
#pragma unroll
                for (int c = 0; c < 3; ++c) o[(size_t)c * N] = f[c];
            }
        } else {
            // Eq. 1's terms with their constants set to 1, of the spins renormalised per site, bonds to +x,
            // +y, +z counted once, and the squared norm of the dipole convolution.  In the path's
            // precision R: the FP64 path sums FP64 terms; the FP32 path's evaluation (its energies only
            // select the images the FP64 evaluation computes, and bound their own round-off) keeps the
            // terms in FP32 and sums them per thread in FP32 and across warps in FP64
            using R = T;
            auto nrm = [](const T* v, R* o) {
                const R a = v[0], b = v[1], c = v[2];
                const R n2 = a * a + b * b + c * c;
                R r = R(0);
                if constexpr (std::is_same<T, float>::value)
                    r = n2 > 0.f ? rsqrtf(n2) : 0.f;
                else
                    r = n2 > 0.0 ? rsqrt_nr(n2) : 0.0;
                o[0] = a * r;
                o[1] = b * r;
                o[2] = c * r;
            };
            R si[3], sx[3], sy[3], sz[3];
            nrm(s0, si);
            R tJ = R(0), tD = R(0);
            if (x + 1 < nx) {
                nrm(xp, sx);
                tJ -= si[0] * sx[0] + si[1] * sx[1] + si[2] * sx[2];
                tD -= si[2] * sx[0] - si[0] * sx[2];  // (x x z) = -y: -(s_i x s_j)_y
            }
            if (y + 1 < ny) {
                nrm(yp, sy);
                tJ -= si[0] * sy[0] + si[1] * sy[1] + si[2] * sy[2];
                tD += si[1] * sy[2] - si[2] * sy[1];  // (y x z) = +x: (s_i x s_j)_x
            }
            if (z + 1 < nz) {
                nrm(zp, sz);
                tJ -= si[0] * sz[0] + si[1] * sz[1] + si[2] * sz[2];
            }
            const R tK = -si[2] * si[2];
            const R tw_ = R(-0.5) * (conv[0] * si[0] + conv[1] * si[1] + conv[2] * si[2]);
            const R cn = conv[0] * conv[0] + conv[1] * conv[1] + conv[2] * conv[2];
            if constexpr (std::is_same<T, float>::value) {
                facc[kEvalTerms * h + 0] += tJ;
                facc[kEvalTerms * h + 1] += tD;
                facc[kEvalTerms * h + 2] += tK;
                facc[kEvalTerms * h + 3] += tw_;
                facc[kEvalTerms * h + 4] += cn;
            } else {
                acc[kEvalTerms * h + 0] += tJ;
                acc[kEvalTerms * h + 1] += tD;
                acc[kEvalTerms * h + 2] += tK;
                acc[kEvalTerms * h + 3] += tw_;
                acc[kEvalTerms * h + 4] += cn;
            }
            if (hout) {
                T* o = hout + (size_t)im * 3 * N + site;
                o[0] = hf[0];
                o[N] = hf[1];
                o[2 * N] = hf[2];
            }
        }
    }
    if constexpr (MODE == 2 || MODE == 5)
        if (dt == T(0)) return;  // uniform over the grid: no energy partials wanted
    if constexpr (MODE != 1)
        block_reduce_t2d<2>(eacc, acc, red);
    else if constexpr (std::is_same<T, float>::value)
        block_reduce_t2d<NV>(facc, acc, red);
    else
        block_reduce_d<NV>(acc, red);
    if (tid == 0) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        for (int h = 0; h < 2; ++h) {
            const int im = ia + h;
            if (im >= g.n_img) continue;
            if (MODE != 1) {
                g.epart[(size_t)blk * g.n_img + im] = acc[h];  // [block][image]
            } else {
                for (int k = 0; k < kEvalTerms; ++k)
                    g.epart[((size_t)blk * g.n_img + im) * kEvalTerms + k] = acc[kEvalTerms * h + k];
            }
        }
    }
}

// xinv: grid (ceil(ny/ty_c), nz, n_pairs).  Inverse x-transform of the pair's field spectra (the
// tensor spectrum already carries 4 pi / (Px Py)), then per site of both images:
//   h = J sum_nn s_j                                                     (Eq. 3)
//     - D (s_z^{+x} - s_z^{-x}, s_z^{+y} - s_z^{-y}, -s_x^{+x} + s_x^{-x} - s_y^{+y} + s_y^{-y})  (Eq. 4)
//     + 2 K s_z z                                                        (Eq. 5)
//     + w * dipole convolution                                           (Eq. 6)
// MODE 0 (step): e += -(1/2) h.s (Eq. 8), s' = normalise(s + dt (h - (s.h) s)) (Eqs. 10, 13).
// MODE 1 (eval): FP64 energy terms of the FP64-renormalised spins, bonds to +x, +y, +z counted once
//                (Eq. 1): tJ = -sum s_i.s_j, tD = sum (r_ij x z).(s_i x s_j), tK = -sum s_z^2,
//                tw = -(1/2) sum conv.s; optionally the field h.
template <typename T, bool DO_FFT, int MODE, int PX>
__global__ void __launch_bounds__(kMaxThreadsX, kMinBlocksX) xinv_kernel(GroupArgs<T> g, T dt, T* hout) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + g.Px;
    double* red = reinterpret_cast<double*>(buf + (DO_FFT ? 3 * g.ty_c * g.lsx : 0));
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * g.ty_c;
    const int rows = min(g.ty_c, g.ny - y0);
    const int ny = g.ny, nz = g.nz;
    if (g.pair_on && !g.pair_on[p]) return;  // uniform over the CTA
    if (DO_FFT)
        for (int i = tid; i < g.Px; i += nthr) tw[i] = PX > 0 ? g.twxs[i] : g.twx[i];
    griddep_wait();
    griddep_launch_dependents();
    if (DO_FFT) {
        const int Px = PX > 0 ? PX : g.Px;
        const C* inp = g.spec + (size_t)p * Px * 3 * nz * ny;
        for (int kc = tid; kc < Px * 3; kc += nthr) {
            const int kx = kc / 3, c = kc - 3 * kx;
            const C* s = inp + ((size_t)kc * nz + z) * ny + y0;
            C* b = buf + c * rows * g.lsx + fft_pad(kx);
            for (int yy = 0; yy < rows; ++yy) b[yy * g.lsx] = cconj(s[yy]);
        }
        __syncthreads();
        fft_lines_any<PX, false, true>(buf, tw, g.planx, g.lsx, 3 * rows, tid, nthr);
    }
    xinv_sites<T, DO_FFT, MODE>(g, dt, hout, buf, g.lsx, red, p, z, y0, rows, tid, nthr);
}

// xinv for Px = 128 (nx <= 64), ROWS (2, 4 or 8) rows per CTA: the inverse x-transform (a forward
// transform of the conjugate) of the 3*ROWS lines in two register passes, inputs read straight from the
// spectrum (rows fastest across a warp), outputs x < 64 into buf; then the same per-site work as
// xinv_kernel.  Rows past ny (last CTA) are skipped.
template <typename T, int MODE, int ROWS>
__global__ void __launch_bounds__(kMaxThreads128, kMinBlocks128) xinv128_kernel(GroupArgs<T> g, T dt, T* hout) {
    using C = cplx<T>;
    static_assert(16 % ROWS == 0 && ROWS >= 2, "the pass-1 role permutation needs ROWS in {2, 4, 8, 16}");
    constexpr int L = 3 * ROWS, NQ = 16 / ROWS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // L lines of kF128Buf, fft_pad positions
    C* zx = buf + L * kF128Buf;                // exchange buffer
    double* red = reinterpret_cast<double*>(zx + (L + 3) / 4 * 4 * kF128Line);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * ROWS;
    const int rows = min(ROWS, g.ny - y0);
    const size_t kstride = (size_t)3 * g.nz * g.ny;  // between consecutive kx
    const C* inp = g.spec + (size_t)p * 128 * kstride + (size_t)z * g.ny + y0;
    const C* __restrict__ tw = g.t2x;  // pass-1 twiddles of length 128
    griddep_wait();
    griddep_launch_dependents();
    // pass 1: role (c, par, j, yy), yy fastest, then j (n2 a permutation of j that puts a half-warp's
    // stores in distinct banks), so par is uniform across a warp for ROWS >= 4
    for (int r = tid; r < 16 * L; r += nthr) {
        const int t = r / ROWS, yy = r % ROWS;
        if (yy >= rows) continue;
        const int j = t & 7, par = (t >> 3) & 1, c = t >> 4;
        const int n2 = (j % NQ) * (8 / NQ) + j / NQ;
        const C* s = inp + (size_t)n2 * kstride + (size_t)c * g.nz * g.ny + yy;  // kx = 8 n1 + n2
        C u[8], hi[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            u[n1] = cconj(s[(size_t)8 * n1 * kstride]);
            hi[n1] = cconj(s[(size_t)(8 * n1 + 64) * kstride]);
        }
        f128_pass1<true>(u, hi, n2, par, tw, zx + (c * ROWS + yy) * kF128Line);
    }
    __syncthreads();
    for (int r = tid; r < 16 * L; r += nthr) {
        const int k1 = r & 15, line = r >> 4;
        if (line % ROWS >= rows) continue;
        C v[8];
        f128_pass2(v, zx + line * kF128Line, k1);
        C* b = buf + (line / ROWS * rows + line % ROWS) * kF128Buf;  // xinv_sites reads line c*rows + yy
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) b[fft_pad(k1 + 16 * k2)] = v[k2];
    }
    __syncthreads();
    xinv_sites<T, true, MODE>(g, dt, hout, buf, kF128Buf, red, p, z, y0, rows, tid, nthr);
}

// ------------------------------------------------------------------------------------------------
// x kernels for Px = P in {192, 256, 384} (nx <= P/2), FP32: the x-transforms in two register passes
// (ss_fft.cuh) on kX2Rows rows of one layer of an image pair per CTA.  Every role order puts the rows
// fastest across a warp: the spectrum's rows of one (kx, c) are contiguous in global memory, and with
// line strides = 16 / kX2Rows (mod 16) the lanes of a half-warp (kX2Rows rows x 16 / kX2Rows consecutive
// columns or rows of a line) hit distinct shared-memory banks.
// xfwd: the gather (Eq. 12) into x-space lines, pass 1 into the transform lines, pass 2 straight to the
// spectrum spec[p][kx][c][z][y].
template <int P>
__global__ void __launch_bounds__(kX2Threads, 3) xfwd2p_kernel(GroupArgs<float> g) {
    using C = float2;
    constexpr int R2 = P / 16, H = R2 / 2, ROWS = kX2Rows, L = 3 * ROWS, LSX = x2_lsx(P), LB = x2_lb(P);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* xb = reinterpret_cast<C*>(smem_raw);  // line c * ROWS + yy: the pair at x, fft_pad positions
    C* A = xb + L * LB;                       // line c * ROWS + yy: rows of Z
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * ROWS;
    const int rows = min(ROWS, g.ny - y0), nx = g.nx;
    const C* __restrict__ tw = g.twx;  // W_P^k
    const C* __restrict__ t1 = g.t2x;  // pass 1
    griddep_wait();
    griddep_launch_dependents();
    xfwd_gather(g, xb, LB, ROWS, p, z, y0, rows, tid, nthr);
    __syncthreads();
    // pass 1, role (yy, n2, c, par)
    for (int r = tid; r < 2 * R2 * L; r += nthr) {
        const int yy = r % ROWS, q = r / ROWS, n2 = q % R2, q2 = q / R2, c = q2 % 3, par = q2 / 3;
        if (yy >= rows) continue;
        const C* b = xb + (c * ROWS + yy) * LB;
        C u[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) u[j] = R2 * j + n2 < nx ? b[fft_pad(R2 * j + n2)] : make_float2(0.f, 0.f);
        t2_pass1<P>(u, n2, par, t1, A + (c * ROWS + yy) * LSX);
    }
    __syncthreads();
    // pass 2, role (yy, k1, par2, c): X[k1 + 16 (2m + par2)] to the spectrum
    const size_t kstride = (size_t)3 * g.nz * g.ny;  // between consecutive kx
    C* outp = g.spec + (size_t)p * P * kstride + (size_t)z * g.ny + y0;
    for (int r = tid; r < 32 * L; r += nthr) {
        const int yy = r % ROWS, q = r / ROWS, k1 = q & 15, par2 = (q >> 4) & 1, c = q >> 5;
        if (yy >= rows) continue;
        const C* col = A + (c * ROWS + yy) * LSX + k1;
        C a[H];
        t2_col_vals<P, false>(a, [&](int j) { return col[j * kT2Row]; }, k1, par2, tw, tw);
        C* o = outp + (size_t)c * g.nz * g.ny + yy;
#pragma unroll
        for (int m = 0; m < H; ++m) o[(size_t)(k1 + 16 * (2 * m + par2)) * kstride] = a[m];
    }
}

// xinv: pass A straight from the spectrum (conjugated) into the transform lines, pass B into x-space
// lines (fft_pad positions, line c * rows + yy), then the per-site work of xinv_sites in mode MODE.
template <int P, int MODE>
__global__ void __launch_bounds__(kX2Threads, 3) xinv2p_kernel(GroupArgs<float> g, float dt, float* hout) {
    using C = float2;
    constexpr int R2 = P / 16, H = R2 / 2, ROWS = kX2Rows, L = 3 * ROWS, LSX = x2_lsx(P), LB = x2_lb(P);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);  // line c * ROWS + yy: columns of T
    C* xb = A + L * LSX;                     // line c * rows + yy: the field convolution at x
    double* red = reinterpret_cast<double*>(xb + L * LB);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int p = blockIdx.z, z = blockIdx.y, y0 = blockIdx.x * ROWS;
    const int rows = min(ROWS, g.ny - y0), nx = g.nx;
    const size_t kstride = (size_t)3 * g.nz * g.ny;
    const C* inp = g.spec + (size_t)p * P * kstride + (size_t)z * g.ny + y0;
    const C* __restrict__ tw = g.twx;
    const C* __restrict__ ta = g.t2x + P;  // pass A
    griddep_wait();
    griddep_launch_dependents();
    // pass A, role (yy, k1, par2, c): column k1 of the conjugated spectrum line (c, yy)
    for (int r = tid; r < 32 * L; r += nthr) {
        const int yy = r % ROWS, q = r / ROWS, k1 = q & 15, par2 = (q >> 4) & 1, c = q >> 5;
        if (yy >= rows) continue;
        const C* sc = inp + (size_t)c * g.nz * g.ny + yy + (size_t)k1 * kstride;
        C a[H];
        t2_col_vals<P, true>(a, [&](int j) { return cconj(sc[(size_t)16 * j * kstride]); }, k1, par2, tw, ta);
        C* o = A + (c * ROWS + yy) * LSX + k1 + par2 * kT2Row;
#pragma unroll
        for (int m = 0; m < H; ++m) o[2 * m * kT2Row] = a[m];
    }
    __syncthreads();
    // pass B, role (yy, y2, c, par): x = y2 + R2 (2m + par) < nx
    for (int r = tid; r < 2 * R2 * L; r += nthr) {
        const int yy = r % ROWS, q = r / ROWS, y2 = q % R2, q2 = q / R2, c = q2 % 3, par = q2 / 3;
        if (yy >= rows) continue;
        C v[8];
        t2_passB(v, A + (c * ROWS + yy) * LSX, y2, par);
        C* b = xb + (c * rows + yy) * LB;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int x = y2 + R2 * (2 * m + par);
            if (x < nx) b[fft_pad(x)] = v[m];
        }
    }
    __syncthreads();
    xinv_sites<float, true, MODE>(g, dt, hout, xb, LB, red, p, z, y0, rows, tid, nthr);
}

// ------------------------------------------------------------------------------------------------
// arc: grid (n_tiles + 1, n_kchunks, n_str), 256 threads.  Tile CTAs: squared distances
// |sp_k - sp_{k-1}|^2 over their share of the 3N components (Eq. 11), one partial per (string, k,
// tile), summed in T per thread and warp, in FP64 across warps.  The last tile CTA of a string to
// finish (ticket counter; nothing waits on another CTA) then sums the tile partials of every d_k in
// FP64 and tile order, scans them into the arc length s_k (Eq. 11), alpha*_k = s_k / s_{K-1} (Eq. 12),
// and for every interior image k finds the largest j with alpha*_j <= k/(K-1) and t: the
// interpolation table the next xfwd applies.  The extra CTA of each chunk (x = n_tiles) sums the step
// kernel's energy partials of the chunk's images (e_last), off that path.  The counters are back at
// zero when the launch ends.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // lane 0
}

// Ticket: atomic add with release (the calling thread's earlier writes, and those ordered before it by a
// barrier, are visible to whoever acquires the new value) and acquire (the writes released by earlier
// tickets are visible to this thread, and after a barrier to its CTA) semantics at GPU scope.
__device__ __forceinline__ unsigned ticket_acq_rel(unsigned* p) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

template <typename T>
__device__ __noinline__ void arc_finish(const GroupArgs<T>& g, const ArcArgs& a, int str, int K, int img0,
                                        double* alpha, double* wsum);

// Reparametrisation variants in the finisher (s holds the arc lengths s_k).  A climbing image kc
// (0 < kc < K-1) splits the string into the parts [0, kc] and [kc, K-1], each brought to equal arc length
// on its own: knots alpha*_j = (s_j - s_a) / (s_b - s_a) and targets (k - a) / (b - a) in part [a, b]; kc
// keeps its place.  Linear interpolation writes the gather table as on the plain path.  The natural
// cubic spline (second derivative zero at a part's ends) writes the identity table and the weights
// phi_k = sum_q W_kq phi*_q (in T) that spline_apply_kernel applies: with knots x_i = alpha*_{a+i}
// (n = b - a segments of lengths h_i), the second derivatives m = P y solve the tridiagonal system
// h_{i-1} m_{i-1} + 2 (h_{i-1} + h_i) m_i + h_i m_{i+1} = 6 ((y_{i+1} - y_i) / h_i - (y_i - y_{i-1}) / h_{i-1})
// (m_0 = m_n = 0; P column by column, one thread each, by forward elimination and back substitution with
// the shared elimination factors), and on segment [x_j, x_{j+1}] the spline is
// A y_j + B y_{j+1} + C m_j + D m_{j+1} with A = (x_{j+1} - x) / h_j, B = (x - x_j) / h_j,
// C = h_j^2 (A^3 - A) / 6, D = h_j^2 (B^3 - B) / 6.  A part with a zero-length segment takes the linear
// rows instead; images that keep their place get identity rows.  Each knot, segment reciprocal and
// elimination factor is formed once (GB300 issues FP64 division slowly).
template <typename T>
__device__ __noinline__ void arc_finish_variants(const GroupArgs<T>& g, const ArcArgs& a, int str, int K, int img0,
                                                 int kc, const double* s) {
    __shared__ double xs[kArcMaxK];  // knot of image k within its part (kc: 1, the end of part one)
    __shared__ double hh_raw[kSplineMaxK], rh_raw[kSplineMaxK], rden_raw[kSplineMaxK], cp_raw[kSplineMaxK];
    // P of a part of up to a.p_dim - 1 segments stays on chip in the launch's dynamic shared memory (the
    // recurrences along a column are dependent, so each step's latency counts); longer parts use the
    // global scratch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Psm = reinterpret_cast<double*>(smem_raw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const bool split = kc > 0 && kc < K - 1;
    const size_t mk = (size_t)a.maxK;
    T* W = reinterpret_cast<T*>(a.W) + (size_t)str * mk * mk;
    auto part_lo = [&](int k) { return split && k > kc ? kc : 0; };
    auto part_hi = [&](int k) { return split && k <= kc ? kc : K - 1; };
    for (int k = tid; k < K; k += nthr) {
        const int a0 = part_lo(k), b0 = part_hi(k);
        const double L = s[b0] - s[a0];
        xs[k] = L > 0.0 && isfinite(L) ? (s[k] - s[a0]) / L : 0.0;
    }
    __syncthreads();
    // knot j of the part starting at a0 (kc starts part two at 0)
    auto knot = [&](int j, int a0) { return j == a0 ? 0.0 : xs[j]; };
    for (int k = tid; k < K; k += nthr) {
        const int a0 = part_lo(k), b0 = part_hi(k);
        const double L = s[b0] - s[a0];
        const bool keep = !a.reparam || k == 0 || k == K - 1 || (split && k == kc) || !(L > 0.0) || !isfinite(L);
        InterpEntry e;
        e.src0 = e.src1 = img0 + k;
        e.t = 0.0;
        e.tf = 0.f;
        e.omtf = 1.f;
        e.copy = 1;
        e.pad = 0;
        if (!keep && !a.spline) {
            const double ak = (double)(k - a0) / (double)(b0 - a0);
            int j = min(max(k, a0), b0 - 1);  // largest j in [a0, b0 - 1] with knot j <= ak, walking from k
            if (knot(j, a0) <= ak) {
                while (j < b0 - 1 && knot(j + 1, a0) <= ak) ++j;
            } else {
                do --j;
                while (knot(j, a0) > ak);
            }
            const double x0 = knot(j, a0), x1 = knot(j + 1, a0);
            e.src0 = img0 + j;
            e.src1 = img0 + j + 1;
            e.t = (ak - x0) / (x1 - x0);
            e.tf = (float)e.t;
            e.omtf = (float)(1.0 - e.t);
            e.copy = 0;
        }
        const_cast<InterpEntry*>(g.interp)[img0 + k] = e;
        if (a.spline) {
            // identity rows for now; the interior rows of a moving part are rewritten below
            T* wr = W + (size_t)k * mk;
            for (int q = 0; q < K; ++q) wr[q] = q == k ? T(1) : T(0);
            a.wcopy[(size_t)str * mk + k] = keep ? 1 : 0;
        }
    }
    if (!a.spline) return;
    // the spline operator in the path's precision T (its weights are stored in T; FP64 arithmetic is slow
    // on GB300 and buys the FP32 path nothing); knots and targets as computed above
    T* hh = reinterpret_cast<T*>(hh_raw);
    T* rh = reinterpret_cast<T*>(rh_raw);
    T* rden = reinterpret_cast<T*>(rden_raw);
    T* cp = reinterpret_cast<T*>(cp_raw);
    for (int part = 0; part < (split ? 2 : 1); ++part) {
        const int a0 = part == 0 ? 0 : kc, b0 = part == 0 && split ? kc : K - 1, n = b0 - a0;
        const double L = s[b0] - s[a0];
        __syncthreads();  // identity rows written; the shared factors are free
        if (!a.reparam || !(L > 0.0) || !isfinite(L) || n < 2) continue;  // uniform: nothing moves here
        bool pos = true;
        for (int i = tid; i < n; i += nthr) {
            const double hd = knot(a0 + i + 1, a0) - knot(a0 + i, a0);
            hh[i] = T(hd);
            pos = pos && hd > 0.0 && hh[i] > T(0);
            if (pos) rh[i] = T(1) / hh[i];
        }
        const bool ok = __syncthreads_and(pos);
        const bool on_chip = n + 1 <= a.p_dim;
        T* P = on_chip ? reinterpret_cast<T*>(Psm) : reinterpret_cast<T*>(a.P) + (size_t)str * mk * mk;
        const size_t ps = on_chip ? (size_t)a.p_dim : mk;  // column stride
        if (ok && tid == 0) {  // elimination factors of the tridiagonal system (m_0 = m_n = 0 known)
            for (int i = 1; i < n; ++i) {
                const T den = T(2) * (hh[i - 1] + hh[i]) - (i > 1 ? hh[i - 1] * cp[i - 1] : T(0));
                rden[i] = T(1) / den;
                cp[i] = (i < n - 1 ? hh[i] : T(0)) * rden[i];
            }
        }
        __syncthreads();
        if (ok) {
            for (int q = tid; q <= n; q += nthr) {  // column q of P: d m_i / d y_q, i = 1..n-1
                T* pc = P + (size_t)q * ps;
                T d = T(0);
                for (int i = 1; i < n; ++i) {
                    T r = T(0);  // d rhs_i / d y_q
                    if (q == i + 1) r = T(6) * rh[i];
                    if (q == i) r = T(-6) * (rh[i] + rh[i - 1]);
                    if (q == i - 1) r = T(6) * rh[i - 1];
                    d = (r - (i > 1 ? hh[i - 1] * d : T(0))) * rden[i];
                    pc[i] = d;
                }
                for (int i = n - 2; i >= 1; --i) pc[i] -= cp[i] * pc[i + 1];
            }
            __syncthreads();
        }
        for (int k = a0 + 1 + tid; k < b0; k += nthr) {
            const double ak = (double)(k - a0) / (double)n;
            int j = min(k, b0 - 1);
            if (knot(j, a0) <= ak) {
                while (j < b0 - 1 && knot(j + 1, a0) <= ak) ++j;
            } else {
                do --j;
                while (knot(j, a0) > ak);
            }
            const double x0 = knot(j, a0), x1 = knot(j + 1, a0);
            T* wr = W + (size_t)k * mk;
            wr[k] = T(0);
            if (!ok) {
                const double t = (ak - x0) / (x1 - x0);
                wr[j] = T(1.0 - t);
                wr[j + 1] = T(t);
                continue;
            }
            const int jr = j - a0;
            const T h = hh[jr], A = T(x1 - ak) * rh[jr], B = T(ak - x0) * rh[jr];
            const T C = h * h * (A * A * A - A) * T(1.0 / 6.0), D = h * h * (B * B * B - B) * T(1.0 / 6.0);
            for (int q = 0; q <= n; ++q) {
                const T* pc = P + (size_t)q * ps;
                const T mj = jr > 0 ? pc[jr] : T(0), mj1 = jr + 1 < n ? pc[jr + 1] : T(0);
                wr[a0 + q] = (q == jr ? A : T(0)) + (q == jr + 1 ? B : T(0)) + C * mj + D * mj1;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 3) arc_kernel(GroupArgs<T> g, ArcArgs a) {
    __shared__ double red[32 * kArcMaxChunk];
    __shared__ double alpha[kArcMaxK];  // d_k, then s_k, then alpha*_k
    __shared__ double wsum[32];
    __shared__ int s_flag;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int str = blockIdx.z, chunk = blockIdx.y;
    const int K = a.str_K[str], img0 = a.str_img0[str];
    const int n_act = max(1, (K - 2 + a.kchunk) / a.kchunk);  // chunks this string uses (one when K = 1)
    const int k_lo = chunk * a.kchunk;
    const int nd = max(0, min(a.kchunk, K - 1 - k_lo));  // differences (k_lo+i, k_lo+i+1), i < nd
    const int n_tiles = a.n_tiles;
    griddep_wait();
    griddep_launch_dependents();
    if (chunk >= n_act) return;  // uniform over the block
    const size_t sb = (size_t)str * a.maxK;
    if ((int)blockIdx.x == n_tiles) {
        // e_last of the chunk's images from the step kernel's partials
        const int k_hi = chunk == n_act - 1 ? K : k_lo + a.kchunk;
        for (int k = k_lo + warp; k < k_hi; k += nwarp) {
            const double* ep = g.epart + img0 + k;  // [block][image]
            double e = 0.0;
            for (int b = lane; b < g.n_eblk; b += 32) e += ep[(size_t)b * g.n_img];
            e = warp_sum_d(e);
            if (lane == 0) {
                if (!isfinite(e)) atomicOr(g.err, kErrNonFinite);
                a.e_last[sb + k] = e;
            }
        }
        if (!a.climb) return;
        // climbing image: the finisher picks the next one from these energies, so they count too
        __syncthreads();
        if (tid == 0) s_flag = ticket_acq_rel(&a.cnt[str]) == (unsigned)((n_tiles + 1) * n_act - 1);
        __syncthreads();
        if (!s_flag) return;
        arc_finish(g, a, str, K, img0, alpha, wsum);
        return;
    }
    const size_t M = (size_t)3 * g.N;
    const size_t e0 = (size_t)blockIdx.x * a.tile_elems;
    const size_t e1 = min(M, e0 + a.tile_elems);
    T part[kArcMaxChunk];  // the thread's few squared differences per image pair, summed in T first
#pragma unroll
    for (int i = 0; i < kArcMaxChunk; ++i) part[i] = T(0);
    if (nd > 0 && sizeof(T) == 4 && (M & 3) == 0 && (e0 & 3) == 0) {
        // four components per thread and load: 16-byte loads of every image of the chunk up front
        const float4* base = reinterpret_cast<const float4*>(g.sp + (size_t)(img0 + k_lo) * M);
        const size_t M4 = M >> 2;
        for (size_t e4 = (e0 >> 2) + tid; e4 < (e1 + 3) >> 2; e4 += nthr) {
            float4 v[kArcMaxChunk + 1];
#pragma unroll
            for (int i = 0; i <= kArcMaxChunk; ++i)
                if (i <= nd) v[i] = base[e4 + (size_t)i * M4];
#pragma unroll
            for (int i = 0; i < kArcMaxChunk; ++i) {
                if (i < nd) {
                    const float dx = v[i + 1].x - v[i].x, dy = v[i + 1].y - v[i].y;
                    const float dz = v[i + 1].z - v[i].z, dw = v[i + 1].w - v[i].w;
                    part[i] += T(dx * dx + dy * dy + dz * dz + dw * dw);
                }
            }
        }
    } else if (nd > 0) {
        for (size_t e = e0 + tid; e < e1; e += nthr) {
            const T* col = g.sp + (size_t)(img0 + k_lo) * M + e;
            T prev = col[0];
#pragma unroll
            for (int i = 0; i < kArcMaxChunk; ++i) {
                if (i < nd) {
                    const T cur = col[(size_t)(i + 1) * M];
                    const T d = cur - prev;
                    part[i] += d * d;
                    prev = cur;
                }
            }
        }
    }
    // block sum: T within each warp (fixed shuffle tree); warp totals in FP64 by 32 lanes of warp 0 at
    // once, lane (i, q) adding warps q, q+4, ... of difference i, then a two-level tree over q
#pragma unroll
    for (int i = 0; i < kArcMaxChunk; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_down_sync(0xffffffffu, part[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < kArcMaxChunk; ++i) red[warp * kArcMaxChunk + i] = double(part[i]);
    __syncthreads();
    if (warp == 0) {
        static_assert(kArcMaxChunk * 4 == 32, "one lane per (difference, quarter)");
        const int i = lane >> 2, q = lane & 3;
        double v = 0.0;
        for (int w = q; w < nwarp; w += 4) v += red[w * kArcMaxChunk + i];
        v += __shfl_down_sync(0xffffffffu, v, 2);
        v += __shfl_down_sync(0xffffffffu, v, 1);
        if (q == 0 && i < nd) a.dpart[((size_t)str * a.maxK + k_lo + i + 1) * n_tiles + blockIdx.x] = v;
        __syncwarp();
        if (lane == 0)
            s_flag = ticket_acq_rel(&a.cnt[str]) == (unsigned)((n_tiles + (a.climb ? 1 : 0)) * n_act - 1);
    }
    __syncthreads();
    if (!s_flag) return;
    arc_finish(g, a, str, K, img0, alpha, wsum);
}

// The last CTA of a string (every partial it needs is visible after its ticket): distances, arc
// length, and the reparametrisation of the variant in use.
template <typename T>
__device__ __noinline__ void arc_finish(const GroupArgs<T>& g, const ArcArgs& a, int str, int K, int img0,
                                        double* alpha, double* wsum) {
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int n_tiles = a.n_tiles;
    // ---- last tile CTA of the string: d_k for k = 1..K-1 ----
    // 8 lanes per difference (lane = 8 j + l, four differences per warp), lane l summing tiles l, l + 8,
    // ... in order (loads twelve at a time), then a three-level tree over l: few FP64 instructions, as
    // GB300 issues FP64 at a low rate
    if (tid == 0) a.cnt[str] = 0u;  // every tile CTA of the string has counted
    {
        const double* dp = a.dpart + (size_t)str * a.maxK * n_tiles;  // [k][tile]
        const int j = lane >> 3, l = lane & 7;
        for (int k0 = 1 + 4 * warp; k0 < K; k0 += 4 * nwarp) {
            const int k = k0 + j;
            double v = 0.0;
            if (k < K) {
                for (int t0 = l; t0 < n_tiles; t0 += 96) {
                    double x[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const int t = t0 + 8 * q;
                        x[q] = t < n_tiles ? __ldcg(dp + (size_t)k * n_tiles + t) : 0.0;
                    }
                    // fixed pairwise tree (FP64 latency is long on GB300; depth 4 instead of 12)
#pragma unroll
                    for (int q = 0; q < 6; ++q) x[q] = x[2 * q] + x[2 * q + 1];
#pragma unroll
                    for (int q = 0; q < 3; ++q) x[q] = x[2 * q] + x[2 * q + 1];
                    v += (x[0] + x[1]) + x[2];
                }
            }
            v += __shfl_down_sync(0xffffffffu, v, 4);
            v += __shfl_down_sync(0xffffffffu, v, 2);
            v += __shfl_down_sync(0xffffffffu, v, 1);
            if (l == 0 && k < K) {
                if (!isfinite(v)) atomicOr(g.err, kErrNonFinite);
                alpha[k] = sqrt_nr(v);  // d_k (Eq. 11)
            }
        }
    }
    if (tid == 0) alpha[0] = 0.0;
    __syncthreads();
    // ---- arc length, targets, interpolation table ----
    const int per = (K + nthr - 1) / nthr;  // images per thread, <= 4 since K <= kArcMaxK = 4 * 256
    const int kb = tid * per;
    const int nw = ((K + per - 1) / per + 31) >> 5;  // warps holding images
    // s_k = d_1 + ... + d_k (Eq. 11): each thread sums the d of its images; an exclusive scan of those
    // sums (warp shuffles, then the warp totals in order) gives its starting offset
    double dloc[4] = {0.0, 0.0, 0.0, 0.0}, ex = 0.0;
    if (warp < nw) {
        double run = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kb + q;
            if (q < per && k < K) {
                dloc[q] = alpha[k];
                run += dloc[q];
            }
        }
        double v = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        ex = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) ex = 0.0;
        if (lane == 31) wsum[warp] = v;
    }
    if (nw > 1) {  // uniform over the block
        __syncthreads();
        if (tid == 0) {
            double off = 0.0;
            for (int w = 0; w < nw; ++w) {
                const double t = wsum[w];
                wsum[w] = off;
                off += t;
            }
        }
        __syncthreads();
    }
    if (warp < nw) {
        double r = (nw > 1 ? wsum[warp] : 0.0) + ex;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kb + q;
            if (q < per && k < K) {
                r += dloc[q];
                alpha[k] = r;
            }
        }
    }
    __syncthreads();
    const int kcur = a.climb ? a.kc[str] : -1;  // the image that climbed in this iteration
    if (a.spline || (kcur > 0 && kcur < K - 1)) {
        arc_finish_variants(g, a, str, K, img0, kcur, alpha);
    } else {
        const double sK = alpha[K - 1];
        const bool move = a.reparam && sK > 0.0 && isfinite(sK);
        if (move && warp < nw) {
            const double r = rcp_nr(sK);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < per && kb + q < K) alpha[kb + q] *= r;  // alpha*_k = s_k / s_{K-1} (Eq. 12)
        }
        __syncthreads();
        if (warp < nw) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = kb + q;
                if (q >= per || k >= K) continue;
                InterpEntry e;
                e.src0 = img0 + k;
                e.src1 = img0 + k;
                e.t = 0.0;
                e.tf = 0.f;
                e.omtf = 1.f;
                e.copy = 1;
                e.pad = 0;
                if (move && k > 0 && k < K - 1) {
                    const double ak = (double)k / (double)(K - 1);
                    // largest j in [0, K-2] with alpha*_j <= ak (alpha* is non-decreasing; alpha*_0 = 0 <= ak),
                    // walking from j = k: after a few iterations the images are nearly evenly spaced
                    int j = min(k, K - 2);
                    if (alpha[j] <= ak) {
                        while (j < K - 2 && alpha[j + 1] <= ak) ++j;
                    } else {
                        do --j;
                        while (alpha[j] > ak);
                    }
                    e.src0 = img0 + j;
                    e.src1 = img0 + j + 1;
                    e.t = (ak - alpha[j]) * rcp_nr(alpha[j + 1] - alpha[j]);
                    e.tf = (float)e.t;
                    e.omtf = (float)(1.0 - e.t);
                    e.copy = 0;
                }
                const_cast<InterpEntry*>(g.interp)[img0 + k] = e;
            }
        }
    }
    if (a.climb) {
        // the next climbing image: the interior maximum of the energies of the states this iteration
        // started from (lowest index on ties); flags for the next x-inverse launch
        __syncthreads();  // every thread has read a.kc[str]
        if (warp == 0) {
            const double* el = a.e_last + (size_t)str * a.maxK;
            double best = -INFINITY;
            int kbest = K;
            for (int k = 1 + lane; k < K - 1; k += 32) {
                const double e = __ldcg(el + k);
                if (e > best) {  // strictly greater: the lane keeps its lowest index
                    best = e;
                    kbest = k;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int ok = __shfl_down_sync(0xffffffffu, kbest, o);
                if (ob > best || (ob == best && ok < kbest)) {
                    best = ob;
                    kbest = ok;
                }
            }
            kbest = __shfl_sync(0xffffffffu, kbest, 0);
            const int kn = K >= 3 && kbest < K - 1 ? kbest : -1;
            if (lane == 0) a.kc[str] = kn;
            for (int k = lane; k < K; k += 32) a.climb_img[img0 + k] = k == kn;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Adaptive Runge-Kutta evolution of the images (Sec. III: explicit Runge-Kutta with step-size control,
// the Dormand-Prince 5(4) pair).  Per attempt, for each stage i: Y_i = y0 + hs sum_{q<i} a_iq k_q
// (rk_assemble into sp), then the field pipeline with an identity table and the step kernel in force
// mode gives k_i = F(Y_i) (Eq. 13); rk_finish forms y5 = y0 + hs sum b_q k_q and the squared scaled
// error (hs sum (b_q - bhat_q) k_q / (atol + rtol max(|y0|, |y5|)))^2 per tile; rk_control (one CTA per
// ODE system) sums it in a fixed order, accepts when sqrt(mean) <= 1 and picks the next step; rk_commit
// renormalises the accepted y5 into y0 (and into sp once the string's interval is complete).
// The Dormand-Prince 5(4) coefficients (Dormand and Prince, 1980): a (rows = stages), the fifth-order
// weights b and the embedded fourth-order weights bh.
constexpr double kDpA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
constexpr double kDpB[7] = {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0};
constexpr double kDpBh[7] = {5179.0 / 57600.0, 0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                             187.0 / 2100.0, 1.0 / 40.0};

// The Runge-Kutta-Fehlberg 4(5) coefficients (Fehlberg, 1969): a (rows = stages), the fourth-order
// weights b4 (carried forward) and the fifth-order weights b5.
constexpr double kRkfA[6][5] = {{0, 0, 0, 0, 0},
                                {1.0 / 4.0, 0, 0, 0, 0},
                                {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
                                {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
                                {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
                                {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
constexpr double kRkfB4[6] = {25.0 / 216.0, 0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0};
constexpr double kRkfB5[6] = {16.0 / 135.0, 0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

// The pair rounded once to the path's precision (the kernels receive it as a launch argument, so the
// FP32 path does no FP64 arithmetic per element); error weights formed in FP64 first.
template <typename T> DpCoef<T> dp_coefficients(int method) {
    DpCoef<T> c{};
    if (method == 0) {
        c.stages = 7;
        for (int i = 0; i < 7; ++i) {
            for (int j = 0; j < 6; ++j) c.a[i][j] = T(kDpA[i][j]);
            c.b[i] = T(kDpB[i]);
            c.e[i] = T(kDpB[i] - kDpBh[i]);
        }
    } else {
        c.stages = 6;
        for (int i = 0; i < 6; ++i) {
            for (int j = 0; j < 5; ++j) c.a[i][j] = T(kRkfA[i][j]);
            c.b[i] = T(kRkfB4[i]);
            c.e[i] = T(kRkfB5[i] - kRkfB4[i]);
        }
    }
    return c;
}
constexpr int kRkTile = 1024;  // components per CTA of the element-wise Runge-Kutta kernels

// grid (tiles, images), 256 threads
// FP32 with N a multiple of 4: the element-wise Runge-Kutta kernels move float4s, one per thread and
// tile (kRkTile = 4 x 256), so every thread has all of its loads in flight at once
template <typename T> __device__ __forceinline__ bool rk_vec4(const GroupArgs<T>& g) {
    return std::is_same<T, float>::value && (g.N & 3) == 0;
}
__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(256) rk_assemble_kernel(GroupArgs<T> g, RkArgs<T> r) {
    const int im = blockIdx.y;
    const size_t M = (size_t)3 * g.N, base = (size_t)im * M, stride = (size_t)g.n_img * M;
    const RkString& S = r.st[r.img_sys[im]];
    const T hs = S.done ? T(0) : T(S.hs);
    if constexpr (std::is_same<T, float>::value) {
        if (rk_vec4(g)) {
            const size_t e4 = (size_t)blockIdx.x * (kRkTile / 4) + threadIdx.x;
            if (4 * e4 >= M) return;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < STAGE; ++q)
                a = f4_fma(r.dp.a[STAGE][q], reinterpret_cast<const float4*>(r.k + q * stride + base)[e4], a);
            reinterpret_cast<float4*>(g.sp + base)[e4] = f4_fma(hs, a, reinterpret_cast<const float4*>(r.y0 + base)[e4]);
            return;
        }
    }
    const size_t e1 = min(M, (size_t)(blockIdx.x + 1) * kRkTile);
    for (size_t e = (size_t)blockIdx.x * kRkTile + threadIdx.x; e < e1; e += blockDim.x) {
        T a = T(0);
#pragma unroll
        for (int q = 0; q < STAGE; ++q) a += r.dp.a[STAGE][q] * r.k[q * stride + base + e];
        g.sp[base + e] = r.y0[base + e] + hs * a;
    }
}

// grid (tiles, images), 256 threads
template <typename T>
__global__ void __launch_bounds__(256) rk_finish_kernel(GroupArgs<T> g, RkArgs<T> r) {
    __shared__ double red[32];
    const int im = blockIdx.y;
    const size_t M = (size_t)3 * g.N, base = (size_t)im * M, stride = (size_t)g.n_img * M;
    const RkString& S = r.st[r.img_sys[im]];
    const T hs = S.done ? T(0) : T(S.hs);
    const T rtol = T(r.rtol), atol = T(r.atol);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *r.active = 0;  // the controllers set it again
    T v[1] = {T(0)};
    const size_t e1 = min(M, (size_t)(blockIdx.x + 1) * kRkTile);
    if constexpr (std::is_same<T, float>::value) {
        if (rk_vec4(g)) {
            const size_t e4 = (size_t)blockIdx.x * (kRkTile / 4) + threadIdx.x;
            if (4 * e4 < M) {
                float4 b5 = make_float4(0.f, 0.f, 0.f, 0.f), d4 = b5;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    if (q >= r.dp.stages) break;
                    const float4 kq = reinterpret_cast<const float4*>(r.k + q * stride + base)[e4];
                    b5 = f4_fma(r.dp.b[q], kq, b5);
                    d4 = f4_fma(r.dp.e[q], kq, d4);
                }
                const float4 y0 = reinterpret_cast<const float4*>(r.y0 + base)[e4];
                const float4 y5 = f4_fma(hs, b5, y0);
                reinterpret_cast<float4*>(r.y5 + base)[e4] = y5;
                const float q0 = hs * d4.x / (atol + rtol * fmaxf(fabsf(y0.x), fabsf(y5.x)));
                const float q1 = hs * d4.y / (atol + rtol * fmaxf(fabsf(y0.y), fabsf(y5.y)));
                const float q2 = hs * d4.z / (atol + rtol * fmaxf(fabsf(y0.z), fabsf(y5.z)));
                const float q3 = hs * d4.w / (atol + rtol * fmaxf(fabsf(y0.w), fabsf(y5.w)));
                v[0] = (q0 * q0 + q1 * q1) + (q2 * q2 + q3 * q3);
            }
        }
    }
    for (size_t e = rk_vec4(g) ? e1 : (size_t)blockIdx.x * kRkTile + threadIdx.x; e < e1; e += blockDim.x) {
        T b5 = T(0), d4 = T(0);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            if (q >= r.dp.stages) break;  // a six-stage pair leaves k_6 unused (it may hold anything)
            const T kq = r.k[q * stride + base + e];
            b5 += r.dp.b[q] * kq;
            d4 += r.dp.e[q] * kq;
        }
        const T y0 = r.y0[base + e];
        const T y5 = y0 + hs * b5;
        r.y5[base + e] = y5;
        const T sc = atol + rtol * max(fabs(y0), fabs(y5));
        const T q = hs * d4 / sc;
        v[0] += q * q;
    }
    double out[1];
    block_reduce_t2d<1>(v, out, red);
    if (threadIdx.x == 0) r.errp[(size_t)im * r.n_tiles + blockIdx.x] = out[0];
}

// grid (n_sys), 256 threads: the system's error norm sqrt(sum / (3N x its images)) over its partials
// (a fixed order), then the step-size control by thread 0, which also marks *r.active (cleared by
// rk_finish) while the system is inside its interval.  begin != 0 opens a new interval instead (t = 0,
// first step cut to T) and marks every system active.
template <typename T>
__global__ void __launch_bounds__(256) rk_control_kernel(GroupArgs<T> g, RkArgs<T> r, int begin) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const double T_int = r.T_int;
    RkString S = r.st[s];
    if (begin) {
        if (threadIdx.x == 0) {
            S.t = 0.0;
            S.done = 0;
            S.accepted = 0;
            S.attempts = 0;
            S.hs = S.step < T_int ? S.step : T_int;
            r.st[s] = S;
            if (s == 0) *r.active = 1;
        }
        return;
    }
    if (S.done) {  // finished in an earlier attempt: nothing to commit this time (uniform over the CTA)
        if (threadIdx.x == 0 && S.accepted) {
            S.accepted = 0;
            r.st[s] = S;
        }
        return;
    }
    const int n = r.sys_cnt[s] * r.n_tiles;
    const double* ep = r.errp + (size_t)r.sys_img0[s] * r.n_tiles;
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += ep[i];
    block_reduce_d<1>(v, red);
    if (threadIdx.x == 0) {
        const double err = sqrt(v[0] / (3.0 * (double)g.N * (double)r.sys_cnt[s]));
        S.err = err;
        if (++S.attempts > 100000) {
            atomicOr(g.err, kErrStepCollapse);
            S.done = 1;
            S.accepted = 0;
        } else {
            // stages that overflowed (F grows like |s|^3 off the unit sphere) give a non-finite norm:
            // a rejection with the smallest factor
            double fac = !isfinite(err) ? 0.2 : err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
            if (fac < 0.2) fac = 0.2;
            if (err <= 1.0) {
                if (fac > 5.0) fac = 5.0;
                S.t = S.hs == T_int - S.t ? T_int : S.t + S.hs;
                S.accepted = 1;
                ++S.acc;
            } else {
                if (fac > 1.0) fac = 1.0;
                S.accepted = 0;
                ++S.rej;
            }
            S.step = S.hs * fac;
            if (S.t >= T_int)
                S.done = 1;
            else
                S.hs = S.step < T_int - S.t ? S.step : T_int - S.t;
        }
        r.st[s] = S;
        if (!S.done) atomicOr(r.active, 1);
    }
}

// grid (site tiles of 256, images), 256 threads: y0 = normalise(y5) per site where the attempt was
// accepted; also into sp once the string's interval is complete
template <typename T>
__global__ void __launch_bounds__(256) rk_commit_kernel(GroupArgs<T> g, RkArgs<T> r) {
    const int im = blockIdx.y;
    const RkString& S = r.st[r.img_sys[im]];
    if (!S.accepted) return;  // uniform over the CTA
    const int N = g.N;
    if constexpr (std::is_same<T, float>::value) {
        if (rk_vec4(g)) {  // four sites per thread, float4 per component plane
            const int i4 = blockIdx.x * blockDim.x + threadIdx.x;
            if (4 * i4 >= N) return;
            const size_t b4 = ((size_t)im * 3 * N) / 4 + i4, p4 = N / 4;
            const float4 a = reinterpret_cast<const float4*>(r.y5)[b4];
            const float4 b = reinterpret_cast<const float4*>(r.y5)[b4 + p4];
            const float4 c = reinterpret_cast<const float4*>(r.y5)[b4 + 2 * p4];
            const float nx_ = rsqrtf(a.x * a.x + b.x * b.x + c.x * c.x), ny_ = rsqrtf(a.y * a.y + b.y * b.y + c.y * c.y);
            const float nz_ = rsqrtf(a.z * a.z + b.z * b.z + c.z * c.z), nw_ = rsqrtf(a.w * a.w + b.w * b.w + c.w * c.w);
            const float4 o[3] = {make_float4(a.x * nx_, a.y * ny_, a.z * nz_, a.w * nw_),
                                 make_float4(b.x * nx_, b.y * ny_, b.z * nz_, b.w * nw_),
                                 make_float4(c.x * nx_, c.y * ny_, c.z * nz_, c.w * nw_)};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                reinterpret_cast<float4*>(r.y0)[b4 + q * p4] = o[q];
                if (S.done) reinterpret_cast<float4*>(g.sp)[b4 + q * p4] = o[q];
            }
            return;
        }
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const size_t base = (size_t)im * 3 * N + i;
    T v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = r.y5[base + (size_t)c * N];
    const T nr = rsqrt_t<T>(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r.y0[base + (size_t)c * N] = v[c] * nr;
        if (S.done) g.sp[base + (size_t)c * N] = v[c] * nr;
    }
}

// ---- direct dipole sum (SS_DIPOLE_DIRECT) -------------------------------------------------------------
// conv_i = sum_{j != i} (3 (r.s_j) r / r^5 - s_j / r^3), r = r_j - r_i in lattice units: Eq. 6 with the
// tensor of Eq. 7 (its 1/(4 pi) cancels against the 4 pi of w's definition); the x-inverse kernel
// multiplies by w.  grid (ceil(N / 128), n_img), 128 threads, one site i each; the image's spins (from s,
// the gathered state) and their coordinates stream through shared memory in tiles of 128 sites.
template <typename T>
__global__ void __launch_bounds__(128) dipole_direct_kernel(GroupArgs<T> g, T* hdir) {
    __shared__ T sj[3][128];
    __shared__ int xj[128], yj[128], zj[128];
    const int im = blockIdx.y, tid = threadIdx.x, N = g.N, nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * 128 + tid;
    const T* s = g.s + (size_t)im * 3 * N;
    const int xi = i % nx, yi = (i / nx) % ny, zi = i / (nx * ny);
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int t0 = 0; t0 < N; t0 += 128) {
        const int j = t0 + tid;
        __syncthreads();  // the previous tile is consumed
        if (j < N) {
            sj[0][tid] = s[j];
            sj[1][tid] = s[N + j];
            sj[2][tid] = s[2 * N + j];
            xj[tid] = j % nx;
            yj[tid] = (j / nx) % ny;
            zj[tid] = j / (nx * ny);
        }
        __syncthreads();
        const int nt = min(128, N - t0);
        for (int q = 0; q < nt; ++q) {
            const T dx = T(xj[q] - xi), dy = T(yj[q] - yi), dz = T(zj[q] - zi);
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == T(0)) continue;  // j == i
            const T ir = rsqrt_t<T>(r2), ir3 = ir * ir * ir, ir5 = ir3 * ir * ir;
            const T rs3 = T(3) * (dx * sj[0][q] + dy * sj[1][q] + dz * sj[2][q]) * ir5;
            a0 += rs3 * dx - sj[0][q] * ir3;
            a1 += rs3 * dy - sj[1][q] * ir3;
            a2 += rs3 * dz - sj[2][q] * ir3;
        }
    }
    if (i < N) {
        T* o = hdir + (size_t)im * 3 * N + i;
        o[0] = a0;
        o[N] = a1;
        o[2 * N] = a2;
    }
}

// ---- climbing image (Euler step) ------------------------------------------------------------------
// The image kc that climbs this iteration stepped neither in the x-inverse kernel (MODE 3 wrote its force
// F = h - (s.h) s into hc); its step reverses F's component along the string's tangent:
//   tau_i = (s_{kc+1,i} - s_{kc-1,i}) - ((s_{kc+1,i} - s_{kc-1,i}) . s_i) s_i   (states before the step)
//   s_i' = normalise(s_i + dt (F_i - 2 (F.tau) / (tau.tau) tau_i))
// climb_dot: grid (c_tiles, n_str), 256 threads: FP64 partials of F.tau and tau.tau per tile of
// kClimbTile sites.  climb_apply: the same grid; every CTA sums its string's partials in one fixed order
// and steps its sites into sp.  Strings with no climbing image return at once.
template <typename T>
__device__ __forceinline__ void climb_site(const GroupArgs<T>& g, const T* hc, int img, int i, T (&s0)[3], T (&F)[3],
                                           T (&tau)[3]) {
    const size_t M = (size_t)3 * g.N;
    const T* sb = g.s + (size_t)img * M + i;
    const T* fb = hc + (size_t)img * M + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s0[c] = sb[(size_t)c * g.N];
        F[c] = fb[(size_t)c * g.N];
        tau[c] = sb[M + (size_t)c * g.N] - sb[(size_t)c * g.N - M];
    }
    const T ts = tau[0] * s0[0] + tau[1] * s0[1] + tau[2] * s0[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) tau[c] -= ts * s0[c];
}

template <typename T>
__global__ void __launch_bounds__(256) climb_dot_kernel(GroupArgs<T> g, ArcArgs a, const T* hc) {
    __shared__ double red[64];
    const int str = blockIdx.y, K = a.str_K[str], kc = a.kc[str];
    if (!(kc > 0 && kc < K - 1)) return;  // uniform over the CTA
    const int img = a.str_img0[str] + kc;
    T v[2] = {T(0), T(0)};
    const int i1 = min(g.N, (int)(blockIdx.x + 1) * kClimbTile);
    for (int i = blockIdx.x * kClimbTile + threadIdx.x; i < i1; i += blockDim.x) {
        T s0[3], F[3], tau[3];
        climb_site(g, hc, img, i, s0, F, tau);
        v[0] += F[0] * tau[0] + F[1] * tau[1] + F[2] * tau[2];
        v[1] += tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    }
    double out[2];
    block_reduce_t2d<2>(v, out, red);
    if (threadIdx.x == 0) {
        double* cp = a.cpart + ((size_t)str * a.c_tiles + blockIdx.x) * 2;
        cp[0] = out[0];
        cp[1] = out[1];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) climb_apply_kernel(GroupArgs<T> g, ArcArgs a, const T* hc, T dt) {
    __shared__ double coef;
    const int str = blockIdx.y, K = a.str_K[str], kc = a.kc[str];
    if (!(kc > 0 && kc < K - 1)) return;  // uniform over the CTA
    const int img = a.str_img0[str] + kc;
    if (threadIdx.x < 32) {
        const double* cp = a.cpart + (size_t)str * a.c_tiles * 2;
        double ft = 0.0, tt = 0.0;
        for (int t = threadIdx.x; t < a.c_tiles; t += 32) {
            ft += cp[2 * t];
            tt += cp[2 * t + 1];
        }
        ft = warp_sum_d(ft);
        tt = warp_sum_d(tt);
        if (threadIdx.x == 0) coef = tt > 0.0 ? ft / tt : 0.0;
    }
    __syncthreads();
    const T c2 = T(2.0 * coef);
    const int N = g.N;
    const int i1 = min(N, (int)(blockIdx.x + 1) * kClimbTile);
    for (int i = blockIdx.x * kClimbTile + threadIdx.x; i < i1; i += blockDim.x) {
        T s0[3], F[3], tau[3], u[3];
        climb_site(g, hc, img, i, s0, F, tau);
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = s0[c] + dt * (F[c] - c2 * tau[c]);
        const T r = rsqrt_t<T>(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        T* o = g.sp + (size_t)img * 3 * N + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) o[(size_t)c * N] = u[c] * r;
    }
}

// ---- natural cubic spline: phi_k = normalise(sum_q W_kq phi*_q) in place on sp -----------------------
// grid (ceil(N / 32), n_str), 256 threads: 32 sites x 8 groups of output rows (row k to group k % 8).
// Dynamic shared memory: the string's K images at the CTA's 32 sites, [K][3][32], then W [K][K] when
// w_on_chip (else W is read through L1).  The tile is loaded whole before any row is written back.
template <typename T>
__global__ void __launch_bounds__(256) spline_apply_kernel(GroupArgs<T> g, ArcArgs a, int w_on_chip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* y = reinterpret_cast<T*>(smem_raw);
    const int str = blockIdx.y, tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    const int K = a.str_K[str], img0 = a.str_img0[str], N = g.N;
    const size_t M = (size_t)3 * N, mk = (size_t)a.maxK;
    const int* wc = a.wcopy + (size_t)str * mk;
    const T* Wg = reinterpret_cast<const T*>(a.W) + (size_t)str * mk * mk;
    T* Ws = y + (size_t)K * 96;
    const int i0 = blockIdx.x * 32, i = i0 + lane;
    for (int e = tid; e < K * 96; e += 256) {  // (q, c, site): 32 consecutive sites per warp load
        const int q = e / 96, r = e - 96 * q, c = r >> 5, l = r & 31;
        y[e] = i0 + l < N ? g.sp[(size_t)(img0 + q) * M + (size_t)c * N + i0 + l] : T(0);
    }
    if (w_on_chip)
        for (int e = tid; e < K * K; e += 256) Ws[e] = Wg[(size_t)(e / K) * mk + e % K];
    __syncthreads();
    if (i >= N) return;
    for (int k = 1 + grp; k < K - 1; k += 8) {
        if (wc[k]) continue;  // kept in place
        T u[3] = {T(0), T(0), T(0)};
        const T* wr = w_on_chip ? Ws + (size_t)k * K : Wg + (size_t)k * mk;
        for (int q = 0; q < K; ++q) {
            const T w = wr[q];
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c] += w * y[q * 96 + c * 32 + lane];
        }
        const T r = rsqrt_t<T>(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        T* o = g.sp + (size_t)(img0 + k) * M + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) o[(size_t)c * N] = u[c] * r;
    }
}

// eval reduce: grid (n_str), thread per image: terms[str][k][4], energies[str][k] and (when cnorm2 is
// given) the squared norm of the dipole convolution cnorm2[str][k], in FP64.  Images of pairs that
// g.pair_on leaves out are skipped (their partials were not written).
template <typename T>
__global__ void eval_reduce_kernel(GroupArgs<T> g, ArcArgs a, double* terms, double* energies, double* cnorm2) {
    const int str = blockIdx.x;
    const int K = a.str_K[str], img0 = a.str_img0[str];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int im = img0 + k;
        if (g.pair_on && !g.pair_on[im >> 1]) continue;
        double t[kEvalTerms];
        for (int q = 0; q < kEvalTerms; ++q) {
            double v = 0.0;
            const double* ep = g.epart + (size_t)im * kEvalTerms + q;
            for (int b = 0; b < g.n_eblk; ++b) v += ep[(size_t)b * g.n_img * kEvalTerms];
            t[q] = v;
            if (q < 4) terms[((size_t)str * a.maxK + k) * 4 + q] = v;
        }
        if (cnorm2) cnorm2[(size_t)str * a.maxK + k] = t[4];
        const ImgParam<T> pr = g.prm[im];
        const double e = (double)pr.J * t[0] + (double)pr.D * t[1] + (double)pr.K * t[2] + (double)pr.w * t[3];
        energies[(size_t)str * a.maxK + k] = e;
        if (!isfinite(e)) atomicOr(g.err, kErrNonFinite);
    }
}

// ------------------------------------------------------------------------------------------------
// layout conversion: caller [K][N][3] <-> internal [K][3][N]; input spins normalised in FP64.
template <typename T, typename Tin>
__global__ void aos_to_soa_kernel(const Tin* src, T* dst, int K, int N, int* err) {
    const size_t total = (size_t)K * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i / N, n = i - k * N;
        const double a = src[3 * i], b = src[3 * i + 1], c = src[3 * i + 2];
        const double n2 = a * a + b * b + c * c;
        double r = 0.0;
        if (!(n2 > 0.0) || !isfinite(n2)) {
            atomicOr(err, kErrInvalidSpin);
        } else {
            r = 1.0 / sqrt(n2);
        }
        T* d = dst + k * 3 * N + n;
        d[0] = T(a * r);
        d[N] = T(b * r);
        d[2 * N] = T(c * r);
    }
}

template <typename T, typename Tout>
__global__ void soa_to_aos_kernel(const T* src, Tout* dst, int K, int N, Tout scale) {
    const size_t total = (size_t)K * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i / N, n = i - k * N;
        const T* s = src + k * 3 * N + n;
        dst[3 * i] = scale * Tout(s[0]);
        dst[3 * i + 1] = scale * Tout(s[N]);
        dst[3 * i + 2] = scale * Tout(s[2 * N]);
    }
}

// ------------------------------------------------------------------------------------------------
#ifdef SS_COMMON_LAUNCHERS
// setup: strided FP64 line FFTs (one line per 1..n lines per CTA) and the octant extraction.
__global__ void __launch_bounds__(256) fft_strided_f64_kernel(double2* data, const double2* twg, FftPlan plan, int n_lines, int lines_per_cta,
                                       long elem_stride, int inner_count, long inner_stride, long outer_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* tw = reinterpret_cast<double2*>(smem_raw);
    double2* buf = tw + plan.P;
    const int P = plan.P, tid = threadIdx.x, nthr = blockDim.x;
    const int l0 = blockIdx.x * lines_per_cta;
    const int L = min(lines_per_cta, n_lines - l0);
    for (int i = tid; i < P; i += nthr) tw[i] = twg[i];
    const int LS = fft_line_stride(P);
    for (int it = tid; it < L * P; it += nthr) {
        const int i = it / P, e = it - i * P;
        const int l = l0 + i;
        const long base = (long)(l % inner_count) * inner_stride + (long)(l / inner_count) * outer_stride;
        buf[i * LS + fft_pad(e)] = data[base + e * elem_stride];
    }
    __syncthreads();
    fft_lines(buf, tw, plan, LS, L, tid, nthr);
    for (int it = tid; it < L * P; it += nthr) {
        const int i = it / P, e = it - i * P;
        const int l = l0 + i;
        const long base = (long)(l % inner_count) * inner_stride + (long)(l / inner_count) * outer_stride;
        data[base + e * elem_stride] = buf[i * LS + fft_pad(e)];
    }
}

#endif

// spec [6][nz][Py][Px] complex (component-major) -> dhat [Px/2+1][|dz|*6 + comp][Py/2+1], scaled:
// for one kx the slab is contiguous and a warp over consecutive ky reads consecutive words.
template <typename T>
__global__ void extract_octant_kernel(const double2* spec, T* dhat, int Px, int Py, int nz, double scale) {
    const int hx = Px / 2 + 1, hy = Py / 2 + 1;
    const size_t total = (size_t)hx * hy * nz * 6;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ky = i % hy;
        size_t r = i / hy;
        const int q = r % (nz * 6);
        const int kx = r / (nz * 6);
        const int dz = q / 6, c = q % 6;
        const double2 v = spec[(((size_t)c * nz + dz) * Py + ky) * Px + kx];
        dhat[i] = T(scale * (c >= 4 ? v.y : v.x));
    }
}

#ifdef SS_COMMON_LAUNCHERS
// grid (site tiles of 256, images): [K][3][N] FP32 spins -> the same spins renormalised in FP64 (the
// dipole convolution of the FP64 evaluation then sees unit vectors, as the local terms do); with pair_on,
// only the images of the flagged pairs (the ones the evaluation computes)
__global__ void widen_unit_kernel(const float* __restrict__ src, double* __restrict__ dst, int K, int N,
                                  const int* __restrict__ pair_on) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    for (int k = blockIdx.y; k < K; k += gridDim.y) {
        if (pair_on && !pair_on[k >> 1]) continue;  // uniform over the CTA
        const size_t b = (size_t)k * 3 * N + n;
        const double a0 = src[b], a1 = src[b + N], a2 = src[b + 2 * (size_t)N];
        const double n2 = a0 * a0 + a1 * a1 + a2 * a2;
        const double r = n2 > 0.0 ? rsqrt_nr(n2) : 0.0;
        dst[b] = a0 * r;
        dst[b + N] = a1 * r;
        dst[b + 2 * (size_t)N] = a2 * r;
    }
}

__global__ void interp_identity_kernel(InterpEntry* tab, int img0, int K) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        InterpEntry e;
        e.src0 = e.src1 = img0 + k;
        e.t = 0.0;
        e.tf = 0.f;
        e.omtf = 1.f;
        e.copy = 1;
        tab[img0 + k] = e;
    }
}
#endif

// ------------------------------------------------------------------------------------------------
// launchers
// Launch with programmatic stream serialisation (see griddep_wait); errors surface through
// cudaGetLastError like a <<<>>> launch.
template <typename... KArgs, typename... Args>
static inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// As launch_pdl, with programmatic stream serialisation only when pdl is set.
template <typename... KArgs, typename... Args>
static inline void launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                             Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The two-pass x-inverse kernel in mode MODE when Px is one of its lengths (rows per CTA kX2Rows, set by
// the host); false otherwise.
template <int MODE>
static inline bool launch_xinv2p(const GroupArgs<float>& g, float dt, float* hout, bool pdl, cudaStream_t st) {
    if (!x2p_ok(4, g.Px)) return false;
    const dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs), blk(kX2Threads);
    const size_t sm = x2_smem(g.Px, true);
    if (g.Px == 192) launch_ex(xinv2p_kernel<192, MODE>, grid, blk, sm, st, pdl, g, dt, hout);
    else if (g.Px == 256) launch_ex(xinv2p_kernel<256, MODE>, grid, blk, sm, st, pdl, g, dt, hout);
    else launch_ex(xinv2p_kernel<384, MODE>, grid, blk, sm, st, pdl, g, dt, hout);
    return true;
}

static inline int grid1d(size_t n, int thr) {
    size_t b = (n + thr - 1) / thr;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b ? b : 1);
}

// Compile-time padded lengths and (Py, nz) pairs of the workloads (FP32 only; the FP64 path and any
// other size use the runtime plans).
#define SS_FOR_PX(X) X(32) X(128) X(192) X(256) X(384)
#define SS_FOR_PYNZ(X) X(32, 1) X(128, 4) X(128, 8) X(192, 4) X(256, 1) X(256, 4) X(256, 8) X(384, 8)
#define SS_FOR_NZ(X) X(1) X(4) X(8)

template <typename T> void launch_xfwd(const GroupArgs<T>& g, bool do_fft, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid((g.ny + g.ty_a - 1) / g.ty_a, g.nz, g.n_pairs);
    if (!do_fft) {
        launch_pdl(xfwd_kernel<T, false, 0>, grid, dim3(nthr), 0, st, g);
        return;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (x2p_ok(4, g.Px)) {  // rows per CTA are kX2Rows (set by the host)
            const size_t sm = x2_smem(g.Px, false);
            if (g.Px == 192) launch_pdl(xfwd2p_kernel<192>, grid, dim3(kX2Threads), sm, st, g);
            else if (g.Px == 256) launch_pdl(xfwd2p_kernel<256>, grid, dim3(kX2Threads), sm, st, g);
            else launch_pdl(xfwd2p_kernel<384>, grid, dim3(kX2Threads), sm, st, g);
            return;
        }
        if (f128_x(4, g.Px)) {
            const dim3 blk(f128_x_threads(g.ty_a));
            const size_t sm = f128_x_smem(g.ty_a);
            if (g.ty_a == 2) launch_pdl(xfwd128_kernel<T, 2>, grid, blk, sm, st, g);
            else if (g.ty_a == 4) launch_pdl(xfwd128_kernel<T, 4>, grid, blk, sm, st, g);
            else launch_pdl(xfwd128_kernel<T, 8>, grid, blk, sm, st, g);  // rows per CTA are 2, 4 or 8
            return;
        }
        switch (g.Px) {
#define SS_CASE(P)                                                \
    case P:                                                       \
        launch_pdl(xfwd_kernel<T, true, P>, grid, dim3(nthr), smem, st, g); \
        return;
            SS_FOR_PX(SS_CASE)
#undef SS_CASE
            default: break;
        }
    }
    launch_pdl(xfwd_kernel<T, true, 0>, grid, dim3(nthr), smem, st, g);
}

template <typename T> void launch_yz(const GroupArgs<T>& g, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid(g.Px, g.n_pairs);
    const size_t base = (size_t)(g.Py + 3 * g.nz * g.lsy) * sizeof(cplx<T>);
    const int stage = smem >= base + (size_t)(g.Py / 2 + 1) * g.nz * 6 * sizeof(T);
    if constexpr (std::is_same<T, float>::value) {
        if (yz2p_ok(4, g.Py, g.nz, g.Px) && g.Px % yz2p_kxb_use(g.nz, g.yz_kxb) == 0) {
            const int kxb = yz2p_kxb_use(g.nz, g.yz_kxb);
            const size_t sm = yz2p_smem(g.Py, g.nz, kxb);
            const dim3 blk(kYz2Threads), gr(g.Px / kxb, g.n_pairs);
#define SS_CASE(P)                                                                         \
    if (g.Py == P) {                                                                       \
        if (g.nz == 1 && kxb == 8) launch_pdl(yz2p_kernel<P, 1, 8>, gr, blk, sm, st, g);      \
        else if (g.nz == 1) launch_pdl(yz2p_kernel<P, 1, 4>, gr, blk, sm, st, g);             \
        else if (g.nz == 4 && kxb == 2) launch_pdl(yz2p_kernel<P, 4, 2>, gr, blk, sm, st, g); \
        else if (g.nz == 4) launch_pdl(yz2p_kernel<P, 4, 1>, gr, blk, sm, st, g);             \
        else launch_pdl(yz2p_kernel<P, 8, 1>, gr, blk, sm, st, g);                            \
        return;                                                                            \
    }
            SS_CASE(192) SS_CASE(256) SS_CASE(384)
#undef SS_CASE
        }
        if (f128_yz(4, g.Py, g.nz)) {
            bool st128 = false;
            const size_t sm128 = f128_yz_smem(g.nz, g.Py, &st128);
            if (g.nz == 8)
                launch_pdl(yz128_kernel<T, 8>, grid, dim3(f128_yz_threads(8)), sm128, st, g, (int)st128);
            else
                launch_pdl(yz128_kernel<T, 4>, grid, dim3(f128_yz_threads(4)), sm128, st, g, (int)st128);
            return;
        }
        if (g.nz == 1 && g.Px % kYzKxb1 == 0) {  // single layer: several kx columns per CTA
            const dim3 gridb(g.Px / kYzKxb1, g.n_pairs);
            const size_t smb = (size_t)(g.Py + 3 * kYzKxb1 * g.lsy) * sizeof(cplx<T>);
            if (g.Py == 256) {
                launch_pdl(yz_kernel<T, 256, 1, kYzKxb1>, gridb, dim3(nthr), smb, st, g, 0);
                return;
            }
            if (g.Py == 32) {
                launch_pdl(yz_kernel<T, 32, 1, kYzKxb1>, gridb, dim3(nthr), smb, st, g, 0);
                return;
            }
        }
        if (g.nz == 4 && g.Px % 2 == 0 && (g.Py == 192 || g.Py == 256)) {  // four layers: two kx columns
            const dim3 gridb(g.Px / 2, g.n_pairs);
            const size_t smb = (size_t)(g.Py + 3 * 4 * 2 * g.lsy) * sizeof(cplx<T>);
            if (g.Py == 192)
                launch_pdl(yz_kernel<T, 192, 4, 2>, gridb, dim3(nthr), smb, st, g, 0);
            else
                launch_pdl(yz_kernel<T, 256, 4, 2>, gridb, dim3(nthr), smb, st, g, 0);
            return;
        }
#define SS_CASE(P, Z)                                                   \
    if (g.Py == P && g.nz == Z) {                                       \
        launch_pdl(yz_kernel<T, P, Z>, grid, dim3(nthr), smem, st, g, stage); \
        return;                                                         \
    }
        SS_FOR_PYNZ(SS_CASE)
#undef SS_CASE
#define SS_CASE(Z)                                                      \
    if (g.nz == Z) {                                                    \
        launch_pdl(yz_kernel<T, 0, Z>, grid, dim3(nthr), smem, st, g, stage); \
        return;                                                         \
    }
        SS_FOR_NZ(SS_CASE)
#undef SS_CASE
    }
    launch_pdl(yz_kernel<T, 0, 0>, grid, dim3(nthr), smem, st, g, stage);
}

template <typename T>
void launch_xinv_step(const GroupArgs<T>& g, bool do_fft, T dt, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs);
    if (!do_fft) {
        launch_pdl(xinv_kernel<T, false, 0, 0>, grid, dim3(nthr), smem, st, g, dt, (T*)nullptr);
        return;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (launch_xinv2p<0>(g, dt, nullptr, true, st)) return;
        if (f128_x(4, g.Px)) {
            const dim3 blk(f128_x_threads(g.ty_c));
            const size_t sm = f128_x_smem(g.ty_c);
            if (g.ty_c == 2) launch_pdl(xinv128_kernel<T, 0, 2>, grid, blk, sm, st, g, dt, (T*)nullptr);
            else if (g.ty_c == 4) launch_pdl(xinv128_kernel<T, 0, 4>, grid, blk, sm, st, g, dt, (T*)nullptr);
            else launch_pdl(xinv128_kernel<T, 0, 8>, grid, blk, sm, st, g, dt, (T*)nullptr);
            return;
        }
        switch (g.Px) {
#define SS_CASE(P)                                                            \
    case P:                                                                   \
        launch_pdl(xinv_kernel<T, true, 0, P>, grid, dim3(nthr), smem, st, g, dt, (T*)nullptr); \
        return;
            SS_FOR_PX(SS_CASE)
#undef SS_CASE
            default: break;
        }
    }
    launch_pdl(xinv_kernel<T, true, 0, 0>, grid, dim3(nthr), smem, st, g, dt, (T*)nullptr);
}

template <typename T>
void launch_xinv_eval(const GroupArgs<T>& g, bool do_fft, T* hout, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs);
    if constexpr (std::is_same<T, float>::value) {
        if (do_fft && launch_xinv2p<1>(g, T(0), hout, false, st)) return;
        if (do_fft && f128_x(4, g.Px)) {
            const int nt = f128_x_threads(g.ty_c);
            const size_t sm = f128_x_smem(g.ty_c);
            if (g.ty_c == 2) xinv128_kernel<T, 1, 2><<<grid, nt, sm, st>>>(g, T(0), hout);
            else if (g.ty_c == 4) xinv128_kernel<T, 1, 4><<<grid, nt, sm, st>>>(g, T(0), hout);
            else xinv128_kernel<T, 1, 8><<<grid, nt, sm, st>>>(g, T(0), hout);
            return;
        }
    }
    if (do_fft) {
        xinv_kernel<T, true, 1, 0><<<grid, nthr, smem, st>>>(g, T(0), hout);
    } else {
        xinv_kernel<T, false, 1, 0><<<grid, nthr, smem, st>>>(g, T(0), hout);
    }
}

template <typename T, int MODE>
static void launch_xinv_force_mode(const GroupArgs<T>& g, bool do_fft, T* kout, T flag, int nthr, size_t smem,
                                   cudaStream_t st) {
    dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs);
    if constexpr (std::is_same<T, float>::value) {
        if (do_fft && launch_xinv2p<MODE>(g, flag, kout, false, st)) return;
        if (do_fft && f128_x(4, g.Px)) {
            const int nt = f128_x_threads(g.ty_c);
            const size_t sm = f128_x_smem(g.ty_c);
            if (g.ty_c == 2) xinv128_kernel<T, MODE, 2><<<grid, nt, sm, st>>>(g, flag, kout);
            else if (g.ty_c == 4) xinv128_kernel<T, MODE, 4><<<grid, nt, sm, st>>>(g, flag, kout);
            else xinv128_kernel<T, MODE, 8><<<grid, nt, sm, st>>>(g, flag, kout);
            return;
        }
    }
    if (do_fft)
        xinv_kernel<T, true, MODE, 0><<<grid, nthr, smem, st>>>(g, flag, kout);
    else
        xinv_kernel<T, false, MODE, 0><<<grid, nthr, smem, st>>>(g, flag, kout);
}

template <typename T>
void launch_xinv_force(const GroupArgs<T>& g, bool do_fft, T* kout, bool energies, bool llg, int nthr, size_t smem,
                       cudaStream_t st) {
    const T flag = energies ? T(1) : T(0);  // force mode: nonzero asks for the energy partials
    if (llg)
        launch_xinv_force_mode<T, 5>(g, do_fft, kout, flag, nthr, smem, st);
    else
        launch_xinv_force_mode<T, 2>(g, do_fft, kout, flag, nthr, smem, st);
}

template <typename T>
void launch_xinv_step_llg(const GroupArgs<T>& g, bool do_fft, T dt, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs);
    if constexpr (std::is_same<T, float>::value) {
        if (do_fft && launch_xinv2p<4>(g, dt, nullptr, true, st)) return;
        if (do_fft && f128_x(4, g.Px)) {
            const dim3 blk(f128_x_threads(g.ty_c));
            const size_t sm = f128_x_smem(g.ty_c);
            if (g.ty_c == 2) launch_pdl(xinv128_kernel<T, 4, 2>, grid, blk, sm, st, g, dt, (T*)nullptr);
            else if (g.ty_c == 4) launch_pdl(xinv128_kernel<T, 4, 4>, grid, blk, sm, st, g, dt, (T*)nullptr);
            else launch_pdl(xinv128_kernel<T, 4, 8>, grid, blk, sm, st, g, dt, (T*)nullptr);
            return;
        }
    }
    if (do_fft)
        launch_pdl(xinv_kernel<T, true, 4, 0>, grid, dim3(nthr), smem, st, g, dt, (T*)nullptr);
    else
        launch_pdl(xinv_kernel<T, false, 4, 0>, grid, dim3(nthr), smem, st, g, dt, (T*)nullptr);
}

template <typename T>
void launch_xinv_step_climb(const GroupArgs<T>& g, bool do_fft, T dt, T* hc, int nthr, size_t smem, cudaStream_t st) {
    dim3 grid((g.ny + g.ty_c - 1) / g.ty_c, g.nz, g.n_pairs);
    if constexpr (std::is_same<T, float>::value) {
        if (do_fft && launch_xinv2p<3>(g, dt, hc, true, st)) return;
        if (do_fft && f128_x(4, g.Px)) {
            const dim3 blk(f128_x_threads(g.ty_c));
            const size_t sm = f128_x_smem(g.ty_c);
            if (g.ty_c == 2) launch_pdl(xinv128_kernel<T, 3, 2>, grid, blk, sm, st, g, dt, hc);
            else if (g.ty_c == 4) launch_pdl(xinv128_kernel<T, 3, 4>, grid, blk, sm, st, g, dt, hc);
            else launch_pdl(xinv128_kernel<T, 3, 8>, grid, blk, sm, st, g, dt, hc);
            return;
        }
    }
    if (do_fft)
        launch_pdl(xinv_kernel<T, true, 3, 0>, grid, dim3(nthr), smem, st, g, dt, hc);
    else
        launch_pdl(xinv_kernel<T, false, 3, 0>, grid, dim3(nthr), smem, st, g, dt, hc);
}

template <typename T> void launch_dipole_direct(const GroupArgs<T>& g, T* hdir, cudaStream_t st) {
    dipole_direct_kernel<T><<<dim3((g.N + 127) / 128, g.n_img), 128, 0, st>>>(g, hdir);
}

template <typename T> void launch_climb(const GroupArgs<T>& g, const ArcArgs& a, T dt, const T* hc, cudaStream_t st) {
    const dim3 grid(a.c_tiles, a.n_str);
    climb_dot_kernel<T><<<grid, 256, 0, st>>>(g, a, hc);
    climb_apply_kernel<T><<<grid, 256, 0, st>>>(g, a, hc, dt);
}

// The spline apply kernel's shared memory for strings of up to maxK images: the [maxK][3][32] tile, and
// W on chip when both fit in 200 KB.
template <typename T> size_t spline_smem(int maxK, bool* w_on_chip) {
    const size_t tile = (size_t)maxK * 96 * sizeof(T), w = (size_t)maxK * maxK * sizeof(T);
    *w_on_chip = tile + w <= 200 * 1024;
    return *w_on_chip ? tile + w : tile;
}

template <typename T> void launch_spline_apply(const GroupArgs<T>& g, const ArcArgs& a, int maxK, cudaStream_t st) {
    bool on_chip = false;
    const size_t sm = spline_smem<T>(maxK, &on_chip);
    spline_apply_kernel<T><<<dim3((g.N + 31) / 32, a.n_str), 256, sm, st>>>(g, a, on_chip ? 1 : 0);
}

template <typename T> void launch_rk_assemble(const GroupArgs<T>& g, const RkArgs<T>& r, int stage, cudaStream_t st) {
    const dim3 grid(r.n_tiles, g.n_img);
    switch (stage) {
        case 0: rk_assemble_kernel<T, 0><<<grid, 256, 0, st>>>(g, r); break;
        case 1: rk_assemble_kernel<T, 1><<<grid, 256, 0, st>>>(g, r); break;
        case 2: rk_assemble_kernel<T, 2><<<grid, 256, 0, st>>>(g, r); break;
        case 3: rk_assemble_kernel<T, 3><<<grid, 256, 0, st>>>(g, r); break;
        case 4: rk_assemble_kernel<T, 4><<<grid, 256, 0, st>>>(g, r); break;
        case 5: rk_assemble_kernel<T, 5><<<grid, 256, 0, st>>>(g, r); break;
        default: rk_assemble_kernel<T, 6><<<grid, 256, 0, st>>>(g, r); break;
    }
}

template <typename T> void launch_rk_finish(const GroupArgs<T>& g, const RkArgs<T>& r, cudaStream_t st) {
    rk_finish_kernel<T><<<dim3(r.n_tiles, g.n_img), 256, 0, st>>>(g, r);
}

template <typename T>
void launch_rk_control(const GroupArgs<T>& g, const RkArgs<T>& r, int begin, cudaStream_t st) {
    rk_control_kernel<T><<<r.n_sys, 256, 0, st>>>(g, r, begin);
}

template <typename T> void launch_rk_commit(const GroupArgs<T>& g, const RkArgs<T>& r, cudaStream_t st) {
    const int per = std::is_same<T, float>::value && (g.N & 3) == 0 ? 4 : 1;  // sites per thread
    rk_commit_kernel<T><<<dim3((g.N / per + 255) / 256, g.n_img), 256, 0, st>>>(g, r);
}

template <typename T> void launch_arc(const GroupArgs<T>& g, const ArcArgs& a, int nthr, cudaStream_t st) {
    dim3 grid(a.n_tiles + 1, a.n_kchunks, a.n_str);  // + one energy CTA per chunk
    launch_pdl(arc_kernel<T>, grid, dim3(nthr), (size_t)a.p_dim * a.p_dim * sizeof(double), st, g, a);
}

template <typename T>
void launch_eval_reduce(const GroupArgs<T>& g, const ArcArgs& a, double* terms, double* energies, double* cnorm2,
                        cudaStream_t st) {
    eval_reduce_kernel<T><<<a.n_str, 128, 0, st>>>(g, a, terms, energies, cnorm2);
}

template <typename T, typename Tin>
void launch_aos_to_soa(const Tin* src, T* dst, int K, int N, int* err, cudaStream_t st) {
    aos_to_soa_kernel<T, Tin><<<grid1d((size_t)K * N, 256), 256, 0, st>>>(src, dst, K, N, err);
}

template <typename T, typename Tout>
void launch_soa_to_aos(const T* src, Tout* dst, int K, int N, Tout scale, cudaStream_t st) {
    soa_to_aos_kernel<T, Tout><<<grid1d((size_t)K * N, 256), 256, 0, st>>>(src, dst, K, N, scale);
}

template <typename T>
void launch_extract_octant(const double2* spec, T* dhat, int Px, int Py, int nz, double scale, cudaStream_t st) {
    const size_t total = (size_t)(Px / 2 + 1) * (Py / 2 + 1) * nz * 6;
    extract_octant_kernel<T><<<grid1d(total, 256), 256, 0, st>>>(spec, dhat, Px, Py, nz, scale);
}

// Raises the dynamic shared-memory limit of every kernel that stages lines in shared memory to
// `bytes` less the kernel's static shared memory (the two together may not exceed `bytes`).
template <typename F> static inline void set_dyn_smem(F* kernel, int bytes) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes - (int)fa.sharedSizeBytes);
}
template <typename T> void set_smem_limits(int bytes) {
    set_dyn_smem(xfwd_kernel<T, true, 0>, bytes);
    set_dyn_smem(yz_kernel<T, 0, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 0, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 1, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 0, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 1, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 2, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 2, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 3, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 3, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 4, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 4, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, true, 5, 0>, bytes);
    set_dyn_smem(xinv_kernel<T, false, 5, 0>, bytes);
    set_dyn_smem(spline_apply_kernel<T>, 200 * 1024);
    set_dyn_smem(arc_kernel<T>, bytes);
    if constexpr (std::is_same<T, float>::value) {
#define SS_CASE(R)                                  \
    set_dyn_smem(xfwd128_kernel<T, R>, bytes);      \
    set_dyn_smem(xinv128_kernel<T, 0, R>, bytes);   \
    set_dyn_smem(xinv128_kernel<T, 1, R>, bytes);   \
    set_dyn_smem(xinv128_kernel<T, 2, R>, bytes);   \
    set_dyn_smem(xinv128_kernel<T, 3, R>, bytes);   \
    set_dyn_smem(xinv128_kernel<T, 4, R>, bytes);   \
    set_dyn_smem(xinv128_kernel<T, 5, R>, bytes);
        SS_CASE(2) SS_CASE(4) SS_CASE(8)
#undef SS_CASE
        set_dyn_smem(yz128_kernel<T, 4>, bytes);
        set_dyn_smem(yz128_kernel<T, 8>, bytes);
#define SS_CASE(P)                                 \
    set_dyn_smem(xfwd2p_kernel<P>, bytes);         \
    set_dyn_smem(xinv2p_kernel<P, 0>, bytes);      \
    set_dyn_smem(xinv2p_kernel<P, 1>, bytes);      \
    set_dyn_smem(xinv2p_kernel<P, 2>, bytes);      \
    set_dyn_smem(xinv2p_kernel<P, 3>, bytes);      \
    set_dyn_smem(xinv2p_kernel<P, 4>, bytes);      \
    set_dyn_smem(xinv2p_kernel<P, 5>, bytes);      \
    set_dyn_smem(yz2p_kernel<P, 1, 4>, bytes);     \
    set_dyn_smem(yz2p_kernel<P, 4, 1>, bytes);     \
    set_dyn_smem(yz2p_kernel<P, 1, 8>, bytes);     \
    set_dyn_smem(yz2p_kernel<P, 4, 2>, bytes);     \
    set_dyn_smem(yz2p_kernel<P, 8, 1>, bytes);
        SS_CASE(192) SS_CASE(256) SS_CASE(384)
#undef SS_CASE
#define SS_CASE(P)                                  \
    set_dyn_smem(xfwd_kernel<T, true, P>, bytes);   \
    set_dyn_smem(xinv_kernel<T, true, 0, P>, bytes);
        SS_FOR_PX(SS_CASE)
#undef SS_CASE
        set_dyn_smem(yz_kernel<T, 256, 1, kYzKxb1>, bytes);
        set_dyn_smem(yz_kernel<T, 32, 1, kYzKxb1>, bytes);
        set_dyn_smem(yz_kernel<T, 192, 4, 2>, bytes);
        set_dyn_smem(yz_kernel<T, 256, 4, 2>, bytes);
#define SS_CASE(P, Z) set_dyn_smem(yz_kernel<T, P, Z>, bytes);
        SS_FOR_PYNZ(SS_CASE)
#undef SS_CASE
#define SS_CASE(Z) set_dyn_smem(yz_kernel<T, 0, Z>, bytes);
        SS_FOR_NZ(SS_CASE)
#undef SS_CASE
    }
}

#ifdef SS_COMMON_LAUNCHERS
void launch_fft_strided_f64(double2* data, const double2* tw, const FftPlan& plan, int n_lines, long elem_stride,
                            int inner_count, long inner_stride, long outer_stride, cudaStream_t st) {
    const int P = plan.P;  // <= 2048 (validated by the host)
    int nthr = 128;
    while (nthr < 256 && fft_lines_per_pass(nthr, P) < 1) nthr *= 2;
    int lpc = std::max(1, std::min(n_lines, fft_lines_per_pass(nthr, P)));
    const size_t smem = (size_t)(P + lpc * fft_line_stride(P)) * sizeof(double2);
    cudaFuncSetAttribute(fft_strided_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (n_lines + lpc - 1) / lpc;
    fft_strided_f64_kernel<<<grid, nthr, smem, st>>>(data, tw, plan, n_lines, lpc, elem_stride, inner_count,
                                                      inner_stride, outer_stride);
}

void launch_interp_identity(InterpEntry* tab, int img0, int K, cudaStream_t st) {
    interp_identity_kernel<<<(K + 127) / 128, 128, 0, st>>>(tab, img0, K);
}

void launch_widen_unit(const float* src, double* dst, int K, int N, const int* pair_on, cudaStream_t st) {
    widen_unit_kernel<<<dim3((N + 255) / 256, std::min(K, 65535)), 256, 0, st>>>(src, dst, K, N, pair_on);
}
#endif

#define SS_INSTANTIATE(T)                                                                                      \
    template void set_smem_limits<T>(int);                                                                     \
    template void launch_xfwd<T>(const GroupArgs<T>&, bool, int, size_t, cudaStream_t);                        \
    template void launch_yz<T>(const GroupArgs<T>&, int, size_t, cudaStream_t);                                \
    template void launch_xinv_step<T>(const GroupArgs<T>&, bool, T, int, size_t, cudaStream_t);                \
    template void launch_xinv_eval<T>(const GroupArgs<T>&, bool, T*, int, size_t, cudaStream_t);               \
    template void launch_xinv_force<T>(const GroupArgs<T>&, bool, T*, bool, bool, int, size_t, cudaStream_t);  \
    template void launch_xinv_step_llg<T>(const GroupArgs<T>&, bool, T, int, size_t, cudaStream_t);             \
    template void launch_xinv_step_climb<T>(const GroupArgs<T>&, bool, T, T*, int, size_t, cudaStream_t);       \
    template void launch_climb<T>(const GroupArgs<T>&, const ArcArgs&, T, const T*, cudaStream_t);             \
    template void launch_dipole_direct<T>(const GroupArgs<T>&, T*, cudaStream_t);                              \
    template void launch_spline_apply<T>(const GroupArgs<T>&, const ArcArgs&, int, cudaStream_t);              \
    template DpCoef<T> dp_coefficients<T>(int);                                                               \
    template void launch_rk_assemble<T>(const GroupArgs<T>&, const RkArgs<T>&, int, cudaStream_t);             \
    template void launch_rk_finish<T>(const GroupArgs<T>&, const RkArgs<T>&, cudaStream_t);                    \
    template void launch_rk_control<T>(const GroupArgs<T>&, const RkArgs<T>&, int, cudaStream_t);                \
    template void launch_rk_commit<T>(const GroupArgs<T>&, const RkArgs<T>&, cudaStream_t);                    \
    template void launch_arc<T>(const GroupArgs<T>&, const ArcArgs&, int, cudaStream_t);                       \
    template void launch_eval_reduce<T>(const GroupArgs<T>&, const ArcArgs&, double*, double*, double*, cudaStream_t); \
    template void launch_aos_to_soa<T, float>(const float*, T*, int, int, int*, cudaStream_t);                 \
    template void launch_aos_to_soa<T, double>(const double*, T*, int, int, int*, cudaStream_t);               \
    template void launch_soa_to_aos<T, float>(const T*, float*, int, int, float, cudaStream_t);                \
    template void launch_soa_to_aos<T, double>(const T*, double*, int, int, double, cudaStream_t);             \
    template void launch_extract_octant<T>(const double2*, T*, int, int, int, double, cudaStream_t);

}  // namespace ss
