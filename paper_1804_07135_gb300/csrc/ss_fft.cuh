// ss_fft.cuh -- batched complex FFTs of lines held in shared memory (Sec. II-A: the dipole field as a
// zero-padded convolution evaluated with FFTs).
//
// Lines of length P (P = 2^a 3^b) sit in shared memory with stride LS = fft_line_stride(P); element i
// of a line is stored at fft_pad(i) (one padding slot per 16 elements against bank conflicts).  The
// transform is a mixed-radix Stockham autosort FFT (radices 8, 4, 3, 2) done in place: in each stage
// every thread reads its butterflies' inputs into registers, the block synchronises, and the outputs
// are written to their autosorted positions.  Twiddles W_P^k = exp(-2 pi i k / P) come from a table in
// shared memory that the host computed in FP64.  Forward transforms only; an inverse is obtained by
// conjugating on load and on store.
#pragma once
#include "ss_internal.h"

namespace ss {

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// FP32 sums as one paired (two-lane) FP32 instruction each
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmi(C a) { return C{a.y, -a.x}; }

// Size-R forward DFTs in registers.
template <int R, typename C> struct Dft;

template <typename C> struct Dft<2, C> {
    static __device__ __forceinline__ void run(C* v) {
        C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <typename C> struct Dft<3, C> {
    static __device__ __forceinline__ void run(C* v) {
        using R = decltype(v[0].x);
        const R h = R(0.8660254037844386467637231707529362);  // sqrt(3)/2
        C s = cadd(v[1], v[2]);
        C d = csub(v[1], v[2]);
        C m = C{v[0].x - R(0.5) * s.x, v[0].y - R(0.5) * s.y};
        C r = cmi(d);  // -i d
        v[0] = cadd(v[0], s);
        v[1] = C{m.x + h * r.x, m.y + h * r.y};
        v[2] = C{m.x - h * r.x, m.y - h * r.y};
    }
};

template <typename C> struct Dft<4, C> {
    static __device__ __forceinline__ void run(C* v) {
        C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        C c = cadd(v[1], v[3]), d = cmi(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};

template <typename C> struct Dft<8, C> {
    static __device__ __forceinline__ void run(C* v) {
        using R = decltype(v[0].x);
        const R q = R(0.7071067811865475244008443621048490);  // sqrt(2)/2
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, C>::run(e);
        Dft<4, C>::run(o);
        // twiddles W8^k, k = 0..3: 1, (q,-q), -i, (-q,-q)
        C t1 = C{q * (o[1].x + o[1].y), q * (o[1].y - o[1].x)};
        C t2 = cmi(o[2]);
        C t3 = C{q * (o[3].y - o[3].x), -q * (o[3].x + o[3].y)};
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], t1);
        v[5] = csub(e[1], t1);
        v[2] = cadd(e[2], t2);
        v[6] = csub(e[2], t2);
        v[3] = cadd(e[3], t3);
        v[7] = csub(e[3], t3);
    }
};

// Size 6 and 12 by Cooley-Tukey over 3 x 2 and 3 x 4 (n = M n1 + n2, k = k1 + 3 k2 with M = 2 or 4):
// 3-point DFTs over n1 for each n2, the twiddles W_N^{n2 k1}, then 2- or 4-point DFTs over n2.
template <typename C> struct Dft<6, C> {
    static __device__ __forceinline__ void run(C* v) {
        using R = decltype(v[0].x);
        const R h = R(0.8660254037844386467637231707529362);  // sqrt(3)/2
        C a[3] = {v[0], v[2], v[4]}, b[3] = {v[1], v[3], v[5]};
        Dft<3, C>::run(a);
        Dft<3, C>::run(b);
        b[1] = cmul(b[1], C{R(0.5), -h});    // W_6^1
        b[2] = cmul(b[2], C{R(-0.5), -h});   // W_6^2
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            v[k1] = cadd(a[k1], b[k1]);
            v[k1 + 3] = csub(a[k1], b[k1]);
        }
    }
};

template <typename C> struct Dft<12, C> {
    static __device__ __forceinline__ void run(C* v) {
        using R = decltype(v[0].x);
        const R h = R(0.8660254037844386467637231707529362);  // sqrt(3)/2
        C a[4][3];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            a[n2][0] = v[n2];
            a[n2][1] = v[4 + n2];
            a[n2][2] = v[8 + n2];
            Dft<3, C>::run(a[n2]);
        }
        // W_12^{n2 k1}: n2 k1 in {1, 2, 2, 3, 4, 6}
        a[1][1] = cmul(a[1][1], C{h, R(-0.5)});      // W_12^1
        a[1][2] = cmul(a[1][2], C{R(0.5), -h});      // W_12^2
        a[2][1] = cmul(a[2][1], C{R(0.5), -h});      // W_12^2
        a[2][2] = cmul(a[2][2], C{R(-0.5), -h});     // W_12^4
        a[3][1] = cmi(a[3][1]);                      // W_12^3 = -i
        a[3][2] = C{-a[3][2].x, -a[3][2].y};         // W_12^6 = -1
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) {
            C q[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            Dft<4, C>::run(q);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 3 * k2] = q[k2];
        }
    }
};

// Size-R DFTs whose inputs R/2..R-1 are zero (the zero-padded half of a forward transform).
template <int R, typename C> struct DftHalfIn;
template <typename C> struct DftHalfIn<2, C> {
    static __device__ __forceinline__ void run(C* v) { v[1] = v[0]; }
};
template <typename C> struct DftHalfIn<4, C> {
    static __device__ __forceinline__ void run(C* v) {
        const C a = v[0], b = v[1], mb = cmi(v[1]);
        v[0] = cadd(a, b);
        v[1] = cadd(a, mb);
        v[2] = csub(a, b);
        v[3] = csub(a, mb);
    }
};
template <typename C> struct DftHalfIn<8, C> {
    static __device__ __forceinline__ void run(C* v) {
        using R = decltype(v[0].x);
        const R q = R(0.7071067811865475244008443621048490);
        // even part DFT4(x0, x2, 0, 0), odd part DFT4(x1, x3, 0, 0)
        const C x0 = v[0], x1 = v[1], x2 = v[2], x3 = v[3];
        const C m2 = cmi(x2), m3 = cmi(x3);
        const C e0 = cadd(x0, x2), e1 = cadd(x0, m2), e2 = csub(x0, x2), e3 = csub(x0, m2);
        const C o0 = cadd(x1, x3), o1 = cadd(x1, m3), o2 = csub(x1, x3), o3 = csub(x1, m3);
        const C t1 = C{q * (o1.x + o1.y), q * (o1.y - o1.x)};
        const C t2 = cmi(o2);
        const C t3 = C{q * (o3.y - o3.x), -q * (o3.x + o3.y)};
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, t1);
        v[5] = csub(e1, t1);
        v[2] = cadd(e2, t2);
        v[6] = csub(e2, t2);
        v[3] = cadd(e3, t3);
        v[7] = csub(e3, t3);
    }
};

// Host-side plan: radices 8, 4, 2 first (largest first), then 3s.
inline FftPlan fft_make_plan(int P) {
    FftPlan p{};
    p.P = P;
    int a = 0, b = 0, q = P;
    while (q % 2 == 0) q /= 2, ++a;
    while (q % 3 == 0) q /= 3, ++b;
    int n = 0;
    const int n8 = a / 3, rem = a % 3;
    if (rem == 1 && n8 == 0) {
        p.radix[n++] = 2;
    } else {
        const int eights = rem == 1 ? n8 - 1 : n8;
        for (int i = 0; i < eights; ++i) p.radix[n++] = 8;
        if (rem == 1) {
            p.radix[n++] = 4;
            p.radix[n++] = 4;
        }
        if (rem == 2) p.radix[n++] = 4;
    }
    for (int i = 0; i < b; ++i) p.radix[n++] = 3;
    p.nstages = n;
    int ns = 1;
    for (int s = 0; s < n; ++s) {
        const int R = p.radix[s];
        p.q[s] = P / R;
        p.ns[s] = ns;
        p.tw[s] = P / (ns * R);
        p.ns_mask[s] = (ns & (ns - 1)) == 0 ? ns - 1 : -1;
        ns *= R;
    }
    return p;
}

// Elements each thread holds in registers per stage: 8 (9 for radix 3).  Lines are transformed in
// passes of fft_lines_per_pass() lines, so any block of at least P/8 threads can transform any number
// of lines.
template <int R> struct StageCap { static constexpr int B = R == 2 ? 4 : R == 3 ? 3 : R == 4 ? 2 : 1; };
constexpr int kFftElemsPerThread = 8;

__host__ __device__ inline int fft_lines_per_pass(int nthr, int P) { return (nthr * kFftElemsPerThread) / P; }
// Smallest block that can transform lines of length P.
__host__ __device__ inline int fft_min_threads(int P) { return (P + kFftElemsPerThread - 1) / kFftElemsPerThread; }

template <int R, typename C>
__device__ __forceinline__ void fft_stage(C* buf, const C* tw, int LS, int L, int Q, int Ns, int twstep, int ns_mask,
                                          int tid, int nthr) {
    constexpr int B = StageCap<R>::B;
    // butterfly b = tid + i*nthr of the pass: line = b / Q, j = b % Q, advanced without divisions
    int line = tid / Q;
    int j = tid - line * Q;
    const int dl = nthr / Q, dj = nthr - dl * Q;
    C v[B][R];
    int dline[B], de[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        dline[i] = -1;
        de[i] = 0;
        if (line < L) {
            const int jm = ns_mask >= 0 ? (j & ns_mask) : (j % Ns);
            const C* src = buf + line * LS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = src[fft_pad(j + r * Q)];
                if (r > 0) x = cmul(x, tw[jm * r * twstep]);
                v[i][r] = x;
            }
            Dft<R, C>::run(v[i]);
            dline[i] = line * LS;
            de[i] = (j - jm) * R + jm;
        }
        j += dj;
        line += dl;
        if (j >= Q) {
            j -= Q;
            ++line;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (dline[i] >= 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[dline[i] + fft_pad(de[i] + r * Ns)] = v[i][r];
        }
    }
    __syncthreads();
}

// Forward FFT of L lines (stride LS, elements at fft_pad positions) in shared memory.  Must be called
// by every thread of the block, with blockDim.x >= fft_min_threads(P).  Ends synchronised.
template <typename C>
__device__ __forceinline__ void fft_lines(C* buf, const C* tw, const FftPlan& plan, int LS, int L, int tid, int nthr) {
    const int lpp = max(1, fft_lines_per_pass(nthr, plan.P));  // the host guarantees >= 1; never loop forever
    for (int l0 = 0; l0 < L; l0 += lpp) {
        const int nl = min(lpp, L - l0);
        C* b = buf + l0 * LS;
        for (int st = 0; st < plan.nstages; ++st) {
            const int Q = plan.q[st], Ns = plan.ns[st], tws = plan.tw[st], msk = plan.ns_mask[st];
            switch (plan.radix[st]) {
                case 8: fft_stage<8>(b, tw, LS, nl, Q, Ns, tws, msk, tid, nthr); break;
                case 4: fft_stage<4>(b, tw, LS, nl, Q, Ns, tws, msk, tid, nthr); break;
                case 3: fft_stage<3>(b, tw, LS, nl, Q, Ns, tws, msk, tid, nthr); break;
                default: fft_stage<2>(b, tw, LS, nl, Q, Ns, tws, msk, tid, nthr); break;
            }
        }
    }
}

// ---- compile-time plans for the padded lengths the workloads use --------------------------------
// Same radix order and stage constants as fft_make_plan, but known to the compiler, so every index
// of a butterfly is a shift, mask or constant multiply.
__host__ __device__ constexpr int cx_pow(int P, int f) { return P % f == 0 ? 1 + cx_pow(P / f, f) : 0; }
__host__ __device__ constexpr int cx_nstages(int P) {
    return (cx_pow(P, 2) % 3 == 1 && cx_pow(P, 2) / 3 == 0 ? 1
            : cx_pow(P, 2) % 3 == 1                        ? cx_pow(P, 2) / 3 + 1
            : cx_pow(P, 2) % 3 == 2                        ? cx_pow(P, 2) / 3 + 1
                                                           : cx_pow(P, 2) / 3) +
           cx_pow(P, 3);
}
// radix of stage s
__host__ __device__ constexpr int cx_radix(int P, int s) {
    return (cx_pow(P, 2) % 3 == 1 && cx_pow(P, 2) / 3 == 0)
               ? (s == 0 ? 2 : 3)
               : (cx_pow(P, 2) % 3 == 1
                      ? (s < cx_pow(P, 2) / 3 - 1 ? 8 : s < cx_pow(P, 2) / 3 + 1 ? 4 : 3)
                      : (cx_pow(P, 2) % 3 == 2 ? (s < cx_pow(P, 2) / 3 ? 8 : s == cx_pow(P, 2) / 3 ? 4 : 3)
                                               : (s < cx_pow(P, 2) / 3 ? 8 : 3)));
}
__host__ __device__ constexpr int cx_ns(int P, int s) { return s == 0 ? 1 : cx_ns(P, s - 1) * cx_radix(P, s - 1); }

// Offset of stage s's twiddles in the per-stage table: stage s (with ns > 1) holds W_P^{jm*r*tw} at
// [jm][r-1], jm < ns, 1 <= r < R, so a butterfly reads its R-1 twiddles at base + constants.  The
// table has P - radix(0) entries in all (fewer than P).
__host__ __device__ constexpr int cx_tw_off(int P, int s) {
    return s == 0 ? 0 : cx_tw_off(P, s - 1) + (cx_ns(P, s - 1) > 1 ? cx_ns(P, s - 1) * (cx_radix(P, s - 1) - 1) : 0);
}
// True when fft_pad(j + r*Q) - fft_pad(j) does not depend on j (loads at base + constants).
__host__ __device__ constexpr bool cx_load_linear(int Q, int R) {
    for (int j = 0; j < Q; ++j)
        for (int r = 0; r < R; ++r)
            if (fft_pad(j + r * Q) - fft_pad(j) != fft_pad(r * Q)) return false;
    return true;
}
// True when fft_pad(e0 + r*NS) - fft_pad(e0) does not depend on the butterfly (stores at base + constants).
__host__ __device__ constexpr bool cx_store_linear(int P, int R, int NS) {
    for (int j = 0; j < P / R; ++j) {
        const int jm = j % NS, e0 = (j - jm) * R + jm;
        for (int r = 0; r < R; ++r)
            if (fft_pad(e0 + r * NS) - fft_pad(e0) != fft_pad(r * NS)) return false;
    }
    return true;
}

// PIN: inputs r >= R/2 of this stage are zero (first stage of a zero-padded forward transform).
// POUT: only outputs r < R/2 are stored (last stage of a transform read below P/2).
template <int P, int S, bool PIN, bool POUT, int R = cx_radix(P, S), int NS = cx_ns(P, S), typename C>
__device__ __forceinline__ void fft_stage_c(C* buf, const C* tws, int LS, int L, int tid, int nthr) {
    constexpr int B = StageCap<R>::B;
    constexpr int RIN = PIN ? R / 2 : R;    // inputs read
    constexpr int ROUT = POUT ? R / 2 : R;  // outputs stored
    constexpr int Q = P / R;
    constexpr bool LIN_LD = cx_load_linear(Q, R);
    constexpr bool LIN_ST = cx_store_linear(P, R, NS);
    constexpr int TWO = cx_tw_off(P, S);
    C v[B][R];
    int dline[B], de[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int b = tid + i * nthr;
        const int line = b / Q, j = b % Q;
        dline[i] = -1;
        de[i] = 0;
        if (line < L) {
            const int jm = j % NS;
            const C* src = buf + line * LS;
            const C* s0 = src + fft_pad(j);
            const C* w = tws + TWO + jm * (R - 1);
#pragma unroll
            for (int r = 0; r < RIN; ++r) {
                C x = LIN_LD ? s0[fft_pad(r * Q)] : src[fft_pad(j + r * Q)];
                if (NS > 1 && r > 0) x = cmul(x, w[r - 1]);
                v[i][r] = x;
            }
            if constexpr (PIN)
                DftHalfIn<R, C>::run(v[i]);
            else
                Dft<R, C>::run(v[i]);
            dline[i] = line * LS;
            de[i] = (j - jm) * R + jm;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < B; ++i) {
        if (dline[i] >= 0) {
            C* d0 = buf + dline[i] + fft_pad(de[i]);
#pragma unroll
            for (int r = 0; r < ROUT; ++r) {
                if (LIN_ST)
                    d0[fft_pad(r * NS)] = v[i][r];
                else
                    buf[dline[i] + fft_pad(de[i] + r * NS)] = v[i][r];
            }
        }
    }
    __syncthreads();
}

template <int P, int S, bool ZERO_HI_IN, bool HI_OUT_UNUSED, typename C>
__device__ __forceinline__ void fft_stages_c(C* buf, const C* tws, int LS, int L, int tid, int nthr) {
    if constexpr (S < cx_nstages(P)) {
        constexpr int R = cx_radix(P, S);
        constexpr bool pin = ZERO_HI_IN && S == 0 && R != 3;
        constexpr bool pout = HI_OUT_UNUSED && S == cx_nstages(P) - 1 && R != 3;
        fft_stage_c<P, S, pin, pout>(buf, tws, LS, L, tid, nthr);
        fft_stages_c<P, S + 1, ZERO_HI_IN, HI_OUT_UNUSED>(buf, tws, LS, L, tid, nthr);
    }
}

// Forward FFT of L lines of compile-time length P; tws is the per-stage twiddle table.
// ZERO_HI_IN: elements P/2..P-1 of every line are zero on entry (their loads are skipped).
// HI_OUT_UNUSED: only elements 0..P/2-1 of the result are read afterwards (the rest is left stale).
template <int P, bool ZERO_HI_IN = false, bool HI_OUT_UNUSED = false, typename C>
__device__ __forceinline__ void fft_lines_c(C* buf, const C* tws, int LS, int L, int tid, int nthr) {
    const int lpp = max(1, fft_lines_per_pass(nthr, P));
    for (int l0 = 0; l0 < L; l0 += lpp)
        fft_stages_c<P, 0, ZERO_HI_IN, HI_OUT_UNUSED>(buf + l0 * LS, tws, LS, min(lpp, L - l0), tid, nthr);
}

// Host: per-stage twiddle table (see cx_tw_off) of a plan from its flat table w[k] = W_P^k.
template <typename C, typename W> inline void fft_stage_twiddles(const FftPlan& p, const W* w, C* out) {
    int o = 0;
    for (int s = 0; s < p.nstages; ++s) {
        const int R = p.radix[s], Ns = p.ns[s];
        if (Ns == 1) continue;
        for (int jm = 0; jm < Ns; ++jm)
            for (int r = 1; r < R; ++r) {
                const W x = w[(jm * r * p.tw[s]) % p.P];
                out[o++] = C{decltype(C{}.x)(x.x), decltype(C{}.x)(x.y)};
            }
    }
}

// ---- length 128 in two register passes -----------------------------------------------------------
// With n = 8 n1 + n2 and k = k1 + 16 k2 (n1, k1 < 16; n2, k2 < 8) and W = W_128,
//   X[k1 + 16 k2] = sum_{n2} W_8^{n2 k2} W^{n2 k1} Y[n2][k1],   Y[n2][k1] = sum_{n1} W_16^{n1 k1} x[8 n1 + n2].
// Split by the parity of k1 = 2 m + par, the 16-point inner DFT is an 8-point DFT over n1 < 8 of
//   u[n1] = (x[8 n1 + n2] + (-1)^par x[8 n1 + 64 + n2]) W_16^{par n1},
// so a line takes two passes of 8-point DFTs in registers with one exchange through shared memory:
// pass 1, role (n2, par): Z[n2][2m + par] = W^{n2 (2m + par)} DFT8(u)[m];
// pass 2, role k1:        X[k1 + 16 k2] = DFT8(Z[.][k1])[k2].
// A line with a zero upper half (x[n] = 0 for n >= 64) drops the second term of u; a transform read
// only below 64 evaluates k2 < 4 in pass 2 (the other outputs are dead code).
// Exchange buffer Z[line][n2][k1] at line * kF128Line + n2 * kF128N2 + k1 (kF128Line = 1 mod 16, in
// ss_internal.h): the 16 lanes of a half-warp reading 16 consecutive k1 of one line, or writing 8 n2 of
// two consecutive lines (pass-1 roles below), touch 16 distinct bank pairs.
constexpr int kF128N2 = 18;
// Pass-1 role r -> (line, n2, par): n2 = r & 7, then four consecutive lines, then par, so par is uniform
// across a warp; lines are taken in groups of four (callers skip line >= their count).
__device__ __forceinline__ void f128_role1(int r, int& line, int& n2, int& par) {
    n2 = r & 7;
    par = (r >> 5) & 1;
    line = ((r >> 6) << 2) | ((r >> 3) & 3);
}

// a * W_16^J for a compile-time J < 8, W_16 = exp(-2 pi i / 16)
template <int J, typename C> __device__ __forceinline__ C mul_w16(C a) {
    using R = decltype(a.x);
    constexpr double c1 = 0.923879532511286756128183189396788933;  // cos(pi/8)
    constexpr double s1 = 0.382683432365089771728459984030398866;  // sin(pi/8)
    constexpr double h = 0.707106781186547524400844362104849039;   // cos(pi/4)
    if constexpr (J == 0) {
        return a;
    } else if constexpr (J == 4) {
        return cmi(a);
    } else if constexpr (J == 2) {
        return C{R(h) * (a.x + a.y), R(h) * (a.y - a.x)};
    } else if constexpr (J == 6) {
        return C{R(h) * (a.y - a.x), R(-h) * (a.x + a.y)};
    } else {
        constexpr double cr = J == 1 ? c1 : J == 3 ? s1 : J == 5 ? -s1 : -c1;
        constexpr double ci = J == 1 ? -s1 : J == 3 ? -c1 : J == 5 ? -c1 : -s1;
        return cmul(a, C{R(cr), R(ci)});
    }
}
template <typename C> __device__ __forceinline__ void mul_w16_ramp(C (&u)[8]) {
    u[1] = mul_w16<1>(u[1]);
    u[2] = mul_w16<2>(u[2]);
    u[3] = mul_w16<3>(u[3]);
    u[4] = mul_w16<4>(u[4]);
    u[5] = mul_w16<5>(u[5]);
    u[6] = mul_w16<6>(u[6]);
    u[7] = mul_w16<7>(u[7]);
}

// Pass 1 for role (n2, par) of one line.  u holds x[8 n1 + n2] for n1 < 8 on entry; hi (when given)
// holds x[8 n1 + 64 + n2].  Writes Z[n2][2m + par] of the line at zl = exchange buffer + line offset.
// t1: the pass-1 twiddle table (GroupArgs::t2x / t2y), W_128^{n2 (2m + par)} at (2m + par) * 8 + n2.
template <bool HAS_HI, typename C>
__device__ __forceinline__ void f128_pass1(C (&u)[8], const C (&hi)[8], int n2, int par, const C* __restrict__ t1,
                                           C* zl) {
    if constexpr (HAS_HI) {
#pragma unroll
        for (int j = 0; j < 8; ++j) u[j] = par ? csub(u[j], hi[j]) : cadd(u[j], hi[j]);
    }
    if (par) mul_w16_ramp(u);
    Dft<8, C>::run(u);
    C* z = zl + n2 * kF128N2 + par;
#pragma unroll
    for (int m = 0; m < 8; ++m) z[2 * m] = cmul(u[m], t1[(2 * m + par) * 8 + n2]);  // W_128^{n2 (2m + par)}
}

// Pass 2 for role k1 of one line: v[k2] = X[k1 + 16 k2] (k2 < KOUT) from Z[.][k1] at zl + k1.
template <typename C> __device__ __forceinline__ void f128_pass2(C (&v)[8], const C* zl, int k1) {
    const C* z = zl + k1;
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = z[n2 * kF128N2];
    Dft<8, C>::run(v);
}

// ---- lengths P = 16 R2 (R2 = 12, 16, 24: 192, 256, 384) in two register passes ------------------------
// A line of P elements is held in shared memory as R2 rows of 16 at row stride kT2Row = 17 (element
// (r, c) at r * 17 + c; a line takes kT2Row * R2 slots).  With n = R2 n1 + n2, k = k1 + 16 k2 (n1, k1 < 16;
// n2, k2 < R2) the forward transform is
//   X[k1 + 16 k2] = sum_{n2} W_R2^{n2 k2} Z[n2][k1],   Z[n2][k1] = W_P^{n2 k1} sum_{n1} W_16^{n1 k1} x[R2 n1 + n2],
// both sums split by the parity of their output index into half-size DFTs (W = W_P, as for length 128):
// pass 1, role (n2, par), inputs x[R2 n1 + n2]: an 8-point DFT of (x[R2 j + n2] +- x[R2 (j+8) + n2]) W_16^{j par}
//   -> row n2 of Z (k1 = 2m + par);
// pass 2, role (k1, par2), column k1 of Z: an R2/2-point DFT of (Z[j][k1] +- Z[j + R2/2][k1]) W_R2^{j par2}
//   -> X[k1 + 16 (2m + par2)], written back in place into column k1 (row k2), so X[ky] sits at
//   (ky >> 4) * 17 + (ky & 15).
// The inverse direction (a forward transform of the conjugate) starts from that column layout: with
// y = y2 + R2 y1,
//   Y[y2 + R2 y1] = sum_{k1} W_16^{k1 y1} T[k1][y2],   T[k1][y2] = W_P^{k1 y2} sum_{k2} W_R2^{k2 y2} V[k1 + 16 k2];
// pass A, role (k1, par2), column k1: the R2/2-point DFTs as in pass 2, times W_P^{k1 y2}, back into column k1
//   (row y2);
// pass B, role (y2, par), row y2: an 8-point DFT of (T[j][y2] +- T[j+8][y2]) W_16^{j par} -> Y[y2 + R2 (2m + par)];
// an inverse read below P/2 keeps m < 4.  The twiddles of pass 1 and pass A come from the tables of
// GroupArgs::t2x / t2y (t1 = the pass-1 half, ta = the pass-A half, indexed so that a warp's lanes read
// consecutive entries); the ramp W_R2^j = W_P^{16 j} from the flat table tw (the same entry across a warp).
__device__ __forceinline__ int t2_at(int r, int c) { return r * kT2Row + c; }
__device__ __forceinline__ int t2_pos(int ky) { return t2_at(ky >> 4, ky & 15); }

// Pass 1 of a line whose upper half is zero: u[j] = x[R2 j + n2] (j < 8) on entry; writes row n2 of Z.
template <int P, typename C>
__device__ __forceinline__ void t2_pass1(C (&u)[8], int n2, int par, const C* __restrict__ t1, C* line) {
    if (par) mul_w16_ramp(u);
    Dft<8, C>::run(u);
#pragma unroll
    for (int m = 0; m < 8; ++m)
        line[t2_at(n2, 2 * m + par)] = cmul(u[m], t1[(2 * m + par) * (P / 16) + n2]);  // W_P^{n2 (2m + par)}
}

// The R2/2-point DFTs of pass 2 (TW_OUT = false) or pass A (TW_OUT = true) for column k1 and parity par2:
// a[m] = the output of row 2m + par2 (times W_P^{k1 (2m + par2)} in pass A).  col(j) returns the column's
// row j (from shared or global memory).
template <int P, bool TW_OUT, typename C, typename Col>
__device__ __forceinline__ void t2_col_vals(C (&a)[P / 32], Col col, int k1, int par2, const C* __restrict__ tw,
                                            const C* __restrict__ ta) {
    constexpr int R2 = P / 16, H = R2 / 2;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const C lo = col(j), hi = col(j + H);
        a[j] = par2 ? csub(lo, hi) : cadd(lo, hi);
    }
    if (par2) {
#pragma unroll
        for (int j = 1; j < H; ++j) a[j] = cmul(a[j], tw[16 * j]);  // W_R2^j
    }
    Dft<H, C>::run(a);
    if constexpr (TW_OUT) {
#pragma unroll
        for (int m = 0; m < H; ++m) a[m] = cmul(a[m], ta[(2 * m + par2) * 16 + k1]);  // W_P^{k1 (2m + par2)}
    }
}

// Pass 2 / pass A in place on a shared line: reads column k1, writes rows 2m + par2 of the same column.
// The caller pairs the roles par2 = 0 and 1 of a column in one warp; the column is read whole before
// either writes (a __syncwarp between the reads and the writes).
template <int P, bool TW_OUT, typename C>
__device__ __forceinline__ void t2_cols(C* line, int k1, int par2, const C* __restrict__ tw, const C* __restrict__ ta) {
    constexpr int H = P / 32;
    C a[H];
    t2_col_vals<P, TW_OUT>(a, [&](int j) { return line[t2_at(j, k1)]; }, k1, par2, tw, ta);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < H; ++m) line[t2_at(2 * m + par2, k1)] = a[m];
}

// Pass B of row y2: v[m] = Y[y2 + R2 (2m + par)] for m < 4 (the outputs below P/2).
template <typename C>
__device__ __forceinline__ void t2_passB(C (&v)[8], const C* line, int y2, int par) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const C lo = line[t2_at(y2, j)], hi = line[t2_at(y2, j + 8)];
        v[j] = par ? csub(lo, hi) : cadd(lo, hi);
    }
    if (par) mul_w16_ramp(v);
    Dft<8, C>::run(v);
}

// Dispatch: compile-time plan when PC > 0 (tw = per-stage table), the runtime plan otherwise (tw =
// flat table).
// The pruning flags apply to the compile-time path only; they require the zero padding / the unread
// outputs to cover at least the upper half of the line (true for padded length 2n when n <= P/2).
template <int PC, bool ZERO_HI_IN = false, bool HI_OUT_UNUSED = false, typename C>
__device__ __forceinline__ void fft_lines_any(C* buf, const C* tw, const FftPlan& plan, int LS, int L, int tid, int nthr) {
    if constexpr (PC > 0)
        fft_lines_c<PC, ZERO_HI_IN, HI_OUT_UNUSED>(buf, tw, LS, L, tid, nthr);
    else
        fft_lines(buf, tw, plan, LS, L, tid, nthr);
}

}  // namespace ss
