// FP32 FFT passes with the length, the radix sequence and the tile shape fixed at compile
// time, for the lattice extents of the hot path. Same Stockham algorithm and data layout as
// the generic kernels in fft.cu (which serve every other length and FP64); here every index
// division is by a constant and the stage loop is unrolled.
//
// Modes:
//   kPlain: unitary FFT of a [outer][N][inner] view along N, src -> dst (may alias);
//           lines of inactive right-hand sides are skipped.
//   kXUpd:  x-axis pass on fermion vectors [nrhs][Nt*L rows][L][4]: x += alpha p,
//           r -= alpha q (written back), partial ||r||^2, forward FFT of r into dst.
//   kXDot:  x-axis inverse FFT of src into dst and partial Re<r, dst>.
//   kTau:   the preconditioner's tau pass (twist, forward FFT, P-hat, inverse FFT, twist).
#include <cmath>

#include "internal.h"
#include "fft_ct.h"

namespace hmc {

struct RadixList {
    int n;
    int r[12];
};

// Stage radices: powers of two in radix-16 stages, the rest of the power of two merged with
// one odd factor where the product stays <= 20, so that most lengths take two stages.
constexpr RadixList radices(int N) {
    RadixList l{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
    int p2 = 1;
    while (N % 2 == 0) { p2 *= 2; N /= 2; }
    int odd[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int no = 0;
    while (N % 5 == 0) { odd[no++] = 5; N /= 5; }
    while (N % 3 == 0) { odd[no++] = 3; N /= 3; }
    while (p2 >= 16) { l.r[l.n++] = 16; p2 /= 16; }
    int first = 0;
    if (p2 > 1) {
        if (no > 0 && p2 * odd[0] <= 20) { l.r[l.n++] = p2 * odd[0]; first = 1; }
        else l.r[l.n++] = p2;
    }
    for (int i = first; i < no; ++i) {
        if (i + 1 < no && odd[i] * odd[i + 1] <= 15) { l.r[l.n++] = odd[i] * odd[i + 1]; ++i; }
        else l.r[l.n++] = odd[i];
    }
    return l;
}

constexpr int kThreads = 256;

// Twiddles known at compile time: cos and sin of 2 pi m / R from their Taylor series on
// [-pi/2, pi/2] (20 terms; the series' own truncation error there is below 1e-20).
constexpr double kPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double ct_sin_series(double x) {
    double t = x, s = x;
    for (int n = 1; n < 20; ++n) { t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0)); s += t; }
    return s;
}
__host__ __device__ constexpr double ct_cos_series(double x) {
    double t = 1.0, s = 1.0;
    for (int n = 1; n < 20; ++n) { t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n)); s += t; }
    return s;
}
__host__ __device__ constexpr double ct_cos2pi(int m, int R) {
    m %= R;
    if (m < 0) m += R;
    double x = 2.0 * kPi * m / R;
    if (x > kPi) x -= 2.0 * kPi;
    if (x > kPi / 2) return -ct_cos_series(kPi - x);
    if (x < -kPi / 2) return -ct_cos_series(-kPi - x);
    return ct_cos_series(x);
}
__host__ __device__ constexpr double ct_sin2pi(int m, int R) {
    m %= R;
    if (m < 0) m += R;
    double x = 2.0 * kPi * m / R;
    if (x > kPi) x -= 2.0 * kPi;
    if (x > kPi / 2) return ct_sin_series(kPi - x);
    if (x < -kPi / 2) return ct_sin_series(-kPi - x);
    return ct_sin_series(x);
}
template <int R> struct TwR { float c[R], s[R]; };   // cos, sin of 2 pi m / R
template <int R> __host__ __device__ constexpr TwR<R> make_tw() {
    TwR<R> t{};
    for (int m = 0; m < R; ++m) { t.c[m] = (float)ct_cos2pi(m, R); t.s[m] = (float)ct_sin2pi(m, R); }
    return t;
}

__device__ __forceinline__ float2 cmulf(float2 a, float c, float s) {   // a * (c + i s)
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// Prime-size DFTs on registers: v[p] <- sum_q v[q] w^{pq}, w = e^{DIR 2 pi i / R}.
template <int R, int DIR>
__device__ __forceinline__ void bfly_prime(float2* v) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else if constexpr (R == 4) {
        const float2 a = v[0], b = v[1], c = v[2], d = v[3];
        const float2 s0 = make_float2(a.x + c.x, a.y + c.y), s1 = make_float2(a.x - c.x, a.y - c.y);
        const float2 s2 = make_float2(b.x + d.x, b.y + d.y), s3 = make_float2(b.x - d.x, b.y - d.y);
        const float2 s3r = make_float2(-DIR * s3.y, DIR * s3.x);   // s3 * (DIR i)
        v[0] = make_float2(s0.x + s2.x, s0.y + s2.y);
        v[2] = make_float2(s0.x - s2.x, s0.y - s2.y);
        v[1] = make_float2(s1.x + s3r.x, s1.y + s3r.y);
        v[3] = make_float2(s1.x - s3r.x, s1.y - s3r.y);
    } else if constexpr (R == 3) {
        // X1,2 = v0 - (v1 + v2)/2 +- DIR i (sqrt3/2)(v1 - v2)
        constexpr float h = (float)ct_sin2pi(1, 3);
        const float2 t1 = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
        const float2 d = make_float2(DIR * h * (v[1].x - v[2].x), DIR * h * (v[1].y - v[2].y));
        const float2 m = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
        v[0] = make_float2(v[0].x + t1.x, v[0].y + t1.y);
        v[1] = make_float2(m.x - d.y, m.y + d.x);
        v[2] = make_float2(m.x + d.y, m.y - d.x);
    } else if constexpr (R == 5) {
        // pairs (1, 4) and (2, 3): X_{1,4} = m1 +- i n1, X_{2,3} = m2 +- i n2
        constexpr float c1 = (float)ct_cos2pi(1, 5), c2 = (float)ct_cos2pi(2, 5);
        constexpr float s1 = (float)ct_sin2pi(1, 5), s2 = (float)ct_sin2pi(2, 5);
        const float2 a1 = make_float2(v[1].x + v[4].x, v[1].y + v[4].y);
        const float2 a2 = make_float2(v[2].x + v[3].x, v[2].y + v[3].y);
        const float2 b1 = make_float2(v[1].x - v[4].x, v[1].y - v[4].y);
        const float2 b2 = make_float2(v[2].x - v[3].x, v[2].y - v[3].y);
        const float2 m1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
        const float2 m2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
        const float2 n1 = make_float2(DIR * (s1 * b1.x + s2 * b2.x), DIR * (s1 * b1.y + s2 * b2.y));
        const float2 n2 = make_float2(DIR * (s2 * b1.x - s1 * b2.x), DIR * (s2 * b1.y - s1 * b2.y));
        v[0] = make_float2(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
        v[1] = make_float2(m1.x - n1.y, m1.y + n1.x);
        v[4] = make_float2(m1.x + n1.y, m1.y - n1.x);
        v[2] = make_float2(m2.x - n2.y, m2.y + n2.x);
        v[3] = make_float2(m2.x + n2.y, m2.y - n2.x);
    } else {
        constexpr TwR<R> T = make_tw<R>();
        float2 out[R];
#pragma unroll
        for (int p = 0; p < R; ++p) {
            float2 acc = v[0];
#pragma unroll
            for (int q = 1; q < R; ++q) {
                const float2 t = cmulf(v[q], T.c[(p * q) % R], DIR * T.s[(p * q) % R]);
                acc.x += t.x;
                acc.y += t.y;
            }
            out[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < R; ++p) v[p] = out[p];
    }
}

// R = R1 * R2 point DFT on registers by one Cooley-Tukey split: with n = n1 + R1 n2 and
// k = k2 + R2 k1, X[k] = sum_n1 w_R1^{n1 k1} w_R^{n1 k2} sum_n2 v[n] w_R2^{n2 k2}.
template <int R1, int R2, int DIR>
__device__ __forceinline__ void bfly_split(float2* v) {
    constexpr int R = R1 * R2;
    constexpr TwR<R> T = make_tw<R>();
    float2 u[R];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
        float2 w[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) w[n2] = v[n1 + R1 * n2];
        bfly_prime<R2, DIR>(w);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
            u[n1 * R2 + k2] = (n1 * k2 == 0) ? w[k2] : cmulf(w[k2], T.c[(n1 * k2) % R], DIR * T.s[(n1 * k2) % R]);
    }
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
        float2 z[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) z[n1] = u[n1 * R2 + k2];
        bfly_prime<R1, DIR>(z);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k2 + R2 * k1] = z[k1];
    }
}

template <int R, int DIR>
__device__ __forceinline__ void bfly(float2* v) {
    if constexpr (R == 2 || R == 3 || R == 4 || R == 5) bfly_prime<R, DIR>(v);
    else if constexpr (R == 6) bfly_split<2, 3, DIR>(v);
    else if constexpr (R == 8) bfly_split<2, 4, DIR>(v);
    else if constexpr (R == 9) bfly_split<3, 3, DIR>(v);
    else if constexpr (R == 10) bfly_split<2, 5, DIR>(v);
    else if constexpr (R == 12) bfly_split<4, 3, DIR>(v);
    else if constexpr (R == 15) bfly_split<3, 5, DIR>(v);
    else if constexpr (R == 16) bfly_split<4, 4, DIR>(v);
    else if constexpr (R == 20) bfly_split<4, 5, DIR>(v);
    else static_assert(R == 2, "unsupported radix");
}

template <int N, int NL, int R, int Ns, int DIR>
__device__ __forceinline__ void stage_ct(const float2* src, float2* dst, const float2* __restrict__ tw) {
    constexpr int M = N / R;
    constexpr int total = M * NL;
    constexpr int tstep = N / (Ns * R);
#pragma unroll 2
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
        const int line = idx % NL, j = idx / NL;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 a = src[(j + r * M) * NL + line];
            if (Ns > 1 && r > 0) {
                float2 w = __ldg(tw + ((r * k * tstep) % N));
                if (DIR > 0) w.y = -w.y;
                a = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
            }
            v[r] = a;
        }
        bfly<R, DIR>(v);
        const int d = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(d + r * Ns) * NL + line] = v[r];
    }
}

// Runs stages S.. of the plan; returns the buffer that holds the result.
template <int N, int NL, int S, int Ns, int DIR>
__device__ __forceinline__ float2* stages_ct(float2* a, float2* b, const float2* __restrict__ tw) {
    constexpr RadixList rl = radices(N);
    if constexpr (S >= rl.n) {
        return a;
    } else {
        constexpr int R = rl.r[S];
        stage_ct<N, NL, R, Ns, DIR>(a, b, tw);
        __syncthreads();
        return stages_ct<N, NL, S + 1, Ns * R, DIR>(b, a, tw);
    }
}

enum { kPlain = 0, kXUpd = 1, kXDot = 2, kTau = 3 };

struct FftcArgs {
    const float2* src;
    float2* dst;
    float2* x;
    float2* r;
    const float2* p;
    const float2* q;
    int64_t outer, inner, opr;   // view [outer][N][inner]; opr = outer indices per RHS
    int64_t nib;                 // inner blocks
    const CgScalars* cgs;
    double* part;
    const float2* tw;
    float scale;
    // kTau: K-hat = e^{i w_n} - 1 - dtau mu_a - 2 dtau t_h cos kx - 2 dtau t_v cos ky (FP32)
    float c0[2], chx[2], chy[2];   // -1 - dtau mu_a, -2 dtau t_h[a], -2 dtau t_v[a]
    int L;
    int bm;   // kTau: inner index = band * 2 L^2 + 2 site + spin (the (x, y) pass's spectrum layout)
    const float* cosk;
    const float2* eitw;
    const float2* twist;
};

// IC = lines along the inner (contiguous) index; OB = NL / IC rows of the outer index.
// Tiles are either IC = 4 (x axis: OB whole rows, contiguous in memory) or IC = NL (y and tau
// axes: one outer index, NL consecutive inner indices). Each thread moves complex pairs
// (16 bytes); all per-element index arithmetic is by compile-time constants.
template <int N, int NL, int IC, int MODE, int DIR>
__global__ void __launch_bounds__(kThreads) k_fftc(FftcArgs A) {
    constexpr int OB = NL / IC;
    constexpr int TOT = N * NL;
    static_assert(IC == 4 || OB == 1, "tile shape");
    static_assert(kThreads % (NL / 2) == 0 && NL % 2 == 0, "line pairs must tile the block");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8];
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* b = a + TOT;

    int64_t o0, i0;
    int k = 0;
    if constexpr (MODE == kXUpd || MODE == kXDot) {
        k = blockIdx.y;
        if (!A.cgs[k].active) return;
        o0 = (int64_t)k * A.opr + (int64_t)blockIdx.x * OB;
        i0 = 0;
    } else {
        o0 = (blockIdx.x / A.nib) * OB;
        i0 = (blockIdx.x % A.nib) * IC;
        if constexpr (IC != 4) {
            if (A.cgs && !A.cgs[o0 / A.opr].active) return;   // one outer index per tile
        }
    }
    float alpha = 0.f;
    if constexpr (MODE == kXUpd) alpha = (float)A.cgs[k].alpha;
    float acc = 0.f;   // per-thread partial, summed in double below

    // ---- load ------------------------------------------------------------------------------
    // IC = 4: the tile is rows [o0, o0 + nrow) of N * 4 contiguous complex numbers.
    // IC = NL: thread owns line pair ic = 2 (tid % (NL/2)) and rows j = tid / (NL/2) + m * JS.
    constexpr int JS = kThreads / (NL / 2);
    int64_t nrow = OB;
    if constexpr (IC == 4) {
        const int64_t oend = (MODE == kXUpd || MODE == kXDot) ? (int64_t)(k + 1) * A.opr : A.outer;
        nrow = min((int64_t)OB, oend - o0);
    }
    const int icp = 2 * (threadIdx.x % (NL / 2));
    const int j0 = threadIdx.x / (NL / 2);
    const bool lane_live = (IC == 4) || (i0 + icp < A.inner);
    if constexpr (IC == 4) {
        const int64_t g0 = o0 * N * 4;
        const int tot = (int)(nrow * N * 4);
        for (int e = 2 * threadIdx.x; e < tot; e += 2 * kThreads) {
            const int c = e & 3, j = (e >> 2) % N, ob = (e >> 2) / N;
            const int64_t g = g0 + e;
            float4 v;
            if constexpr (MODE == kXUpd) {
                float4 xx = *reinterpret_cast<const float4*>(A.x + g);
                float4 rr = *reinterpret_cast<const float4*>(A.r + g);
                const float4 pp = *reinterpret_cast<const float4*>(A.p + g);
                const float4 qq = *reinterpret_cast<const float4*>(A.q + g);
                xx.x += alpha * pp.x; xx.y += alpha * pp.y; xx.z += alpha * pp.z; xx.w += alpha * pp.w;
                rr.x -= alpha * qq.x; rr.y -= alpha * qq.y; rr.z -= alpha * qq.z; rr.w -= alpha * qq.w;
                *reinterpret_cast<float4*>(A.x + g) = xx;
                *reinterpret_cast<float4*>(A.r + g) = rr;
                acc += rr.x * rr.x + rr.y * rr.y + rr.z * rr.z + rr.w * rr.w;
                v = rr;
            } else {
                v = *reinterpret_cast<const float4*>(A.src + g);
            }
            *reinterpret_cast<float4*>(a + j * NL + ob * 4 + c) = v;
        }
        if (nrow < OB) {   // zero the rows past the end (their results are discarded)
            for (int e = (int)(nrow * N * 4) + threadIdx.x; e < OB * N * 4; e += kThreads) {
                const int c = e & 3, j = (e >> 2) % N, ob = (e >> 2) / N;
                a[j * NL + ob * 4 + c] = make_float2(0.f, 0.f);
            }
        }
    } else {
        const float2* src = A.src + (o0 * N + j0) * A.inner + i0 + icp;
        const int64_t step = (int64_t)JS * A.inner;
#pragma unroll 4
        for (int j = j0; j < N; j += JS, src += step) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lane_live) {
                v = *reinterpret_cast<const float4*>(src);
                if constexpr (MODE == kTau) {
                    const float2 w = __ldg(A.twist + j);   // multiply by conj(w)
                    v = make_float4(v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y,
                                    v.z * w.x + v.w * w.y, v.w * w.x - v.z * w.y);
                }
            }
            *reinterpret_cast<float4*>(a + j * NL + icp) = v;
        }
    }
    __syncthreads();

    // ---- transform -------------------------------------------------------------------------
    float2* res;
    if constexpr (MODE == kTau) {
        res = stages_ct<N, NL, 0, 1, -1>(a, b, A.tw);
        float2* other = (res == a) ? b : a;
        // P-hat = 1 / |K-hat|^2: the momentum part depends only on the thread's line pair
        // (both lines share alpha and k: they are spins s = 0, 1 of one site, adjacent in both
        // inner layouts)
        const int64_t i = i0 + icp;
        float base = 0.f;
        if (lane_live) {
            const int64_t half = 2 * (int64_t)A.L * A.L;   // inner indices of one band
            const int ab = A.bm ? (i >= half ? 1 : 0) : (int)((i & 3) >> 1);
            const int kk = A.bm ? (int)((i - ab * half) >> 1) : (int)(i >> 2);
            const int mx = kk % A.L, my = kk / A.L;
            base = A.c0[ab] + A.chx[ab] * __ldg(A.cosk + mx) + A.chy[ab] * __ldg(A.cosk + my);
        }
#pragma unroll 4
        for (int j = j0; j < N; j += JS) {
            const float2 ew = __ldg(A.eitw + j);
            const float re = ew.x + base;
            const float ph = 1.0f / (re * re + ew.y * ew.y);
            float4 v = *reinterpret_cast<float4*>(res + j * NL + icp);
            acc += ph * (v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);   // sum P-hat |v|^2
            v.x *= ph; v.y *= ph; v.z *= ph; v.w *= ph;
            *reinterpret_cast<float4*>(res + j * NL + icp) = v;
        }
        __syncthreads();
        res = stages_ct<N, NL, 0, 1, +1>(res, other, A.tw);
    } else {
        res = stages_ct<N, NL, 0, 1, DIR>(a, b, A.tw);
    }

    // ---- store -----------------------------------------------------------------------------
    const float sc = A.scale;
    if constexpr (IC == 4) {
        const int64_t g0 = o0 * N * 4;
        const int tot = (int)(nrow * N * 4);
        for (int e = 2 * threadIdx.x; e < tot; e += 2 * kThreads) {
            const int c = e & 3, j = (e >> 2) % N, ob = (e >> 2) / N;
            const int64_t g = g0 + e;
            float4 v = *reinterpret_cast<const float4*>(res + j * NL + ob * 4 + c);
            v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
            *reinterpret_cast<float4*>(A.dst + g) = v;
            if constexpr (MODE == kXDot) {
                const float4 rr = *reinterpret_cast<const float4*>(A.r + g);
                acc += rr.x * v.x + rr.y * v.y + rr.z * v.z + rr.w * v.w;
            }
        }
    } else if (lane_live) {
        float2* dst = A.dst + (o0 * N + j0) * A.inner + i0 + icp;
        const int64_t step = (int64_t)JS * A.inner;
#pragma unroll 4
        for (int j = j0; j < N; j += JS, dst += step) {
            float4 v = *reinterpret_cast<const float4*>(res + j * NL + icp);
            if constexpr (MODE == kTau) {
                const float2 w = __ldg(A.twist + j);
                v = make_float4(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x,
                                v.z * w.x - v.w * w.y, v.z * w.y + v.w * w.x);
            }
            v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
            *reinterpret_cast<float4*>(dst) = v;
        }
    }
    if constexpr (MODE == kXUpd || MODE == kXDot) {
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0) A.part[(int64_t)k * gridDim.x + blockIdx.x] = tot;
    }
    if constexpr (MODE == kTau) {
        // the forward FFT above is unnormalised: |v|^2 = N |unitary coefficient|^2
        if (A.part) {
            const double tot = block_sum((double)acc, red);
            if (threadIdx.x == 0) A.part[blockIdx.x] = tot / N;   // block = k * nib + inner block
        }
    }
}

// ---- dispatch ------------------------------------------------------------------------------
template <int N> constexpr int lines_for() { return N > 96 ? 16 : 32; }

template <int N, int IC, int MODE, int DIR>
static int launch_one(hmc_ctx* ctx, dim3 grid, const FftcArgs& A) {
    constexpr int NL = lines_for<N>();
    constexpr int ICr = (IC == 4) ? 4 : NL;
    const size_t sm = 2 * (size_t)N * NL * sizeof(float2);
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fftc<N, NL, ICr, MODE, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm));
        attr.mark(bit);
    }
    k_fftc<N, NL, ICr, MODE, DIR><<<grid, kThreads, sm, ctx->stream>>>(A);
    HMC_LAUNCH(ctx, "k_fftc");
    return HMC_OK;
}

// Lengths with compiled kernels.
#define HMC_FFTC_SIZES(X) X(4) X(6) X(8) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(120) X(128) X(160) X(200)

bool fftc_supported(int n) {
#define HMC_CASE(N) if (n == N) return true;
    HMC_FFTC_SIZES(HMC_CASE)
#undef HMC_CASE
    return false;
}

static int lines_rt(int n) { return n > 96 ? 16 : 32; }

bool fftc_can(int n, int64_t inner) {
    return fftc_supported(n) && (inner == 4 || (inner >= lines_rt(n) && inner % 2 == 0));
}

// Plain axis pass (IC = lines if inner >= lines, else IC = 4 with inner == 4).
int fftc_axis(hmc_ctx* ctx, float2* data, int64_t outer, int n, int64_t inner, int dir, const float2* src,
              const CgScalars* cgs, int64_t opr) {
    const FftPlan* pl = get_plan(ctx, n);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan");
    const int NL = lines_rt(n);
    FftcArgs A{};
    A.src = src ? src : data;
    A.dst = data;
    A.outer = outer;
    A.inner = inner;
    A.opr = opr > 0 ? opr : 1;
    A.cgs = cgs;
    A.tw = pl->tw32;
    A.scale = (float)(1.0 / std::sqrt((double)n));
    const bool x4 = inner == 4;
    if (!x4 && inner < NL) return fail(ctx, HMC_ERR_STATE, "fftc: unsupported tile");
    const int IC = x4 ? 4 : NL, OB = NL / IC;
    A.nib = (inner + IC - 1) / IC;
    const dim3 grid((unsigned)(((outer + OB - 1) / OB) * A.nib));
#define HMC_CASE(N)                                                                          \
    if (n == N) {                                                                            \
        if (x4) return dir < 0 ? launch_one<N, 4, kPlain, -1>(ctx, grid, A)                  \
                               : launch_one<N, 4, kPlain, +1>(ctx, grid, A);                 \
        return dir < 0 ? launch_one<N, 0, kPlain, -1>(ctx, grid, A)                          \
                       : launch_one<N, 0, kPlain, +1>(ctx, grid, A);                         \
    }
    HMC_FFTC_SIZES(HMC_CASE)
#undef HMC_CASE
    return fail(ctx, HMC_ERR_STATE, "fftc: unsupported length");
}

// ---- tau pass in place ------------------------------------------------------------------------
// The preconditioner's tau pass (twist, FFT along tau, P-hat, inverse FFT, twist) for 16
// consecutive inner indices (4 sites x 4 components) of one right-hand side, all N slices in
// one shared buffer [N][16]. The FFT is the same in-place two-factor split as the (x, y) pass,
// N = N1 * N2: the spectrum between the forward and inverse steps is in digit-permuted order
// (position N1 k2 + k1 holds frequency k2 + N2 k1) and P-hat reads e^{i w_n} in that order. The
// forward twist is applied as step A reads its points, the inverse twist as the result is stored.
template <int N> struct TauSplit { static constexpr int N1 = 0, N2 = 0; };
template <> struct TauSplit<4> { static constexpr int N1 = 2, N2 = 2; };
template <> struct TauSplit<6> { static constexpr int N1 = 3, N2 = 2; };
template <> struct TauSplit<8> { static constexpr int N1 = 4, N2 = 2; };
template <> struct TauSplit<12> { static constexpr int N1 = 4, N2 = 3; };
template <> struct TauSplit<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct TauSplit<20> { static constexpr int N1 = 5, N2 = 4; };
template <> struct TauSplit<24> { static constexpr int N1 = 6, N2 = 4; };
template <> struct TauSplit<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct TauSplit<40> { static constexpr int N1 = 8, N2 = 5; };
template <> struct TauSplit<48> { static constexpr int N1 = 8, N2 = 6; };
template <> struct TauSplit<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct TauSplit<80> { static constexpr int N1 = 10, N2 = 8; };
template <> struct TauSplit<160> { static constexpr int N1 = 16, N2 = 10; };
#define HMC_TAU2_SIZES(X) X(4) X(6) X(8) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(80) X(160)

constexpr int kTauLines = 16, kTauThreads = 256;

// The tau pass in three steps over a shared tile [N][16] of one right-hand side's 16
// consecutive inner indices (4 sites x 4 components), N = N1 * N2, loaded whole first:
//   1. (line, n1): the N2 points t = n1 + N1 m of the tile, times
//      conj(e^{i pi t / N}) (the twist), N2-point DFT over m, times w_N^{-n1 k2}, into the tile
//      at position n1 + N1 k2;
//   2. (line, k2): the N1 points at positions N1 k2 + m: N1-point DFT over m (the spectrum, in
//      digit-permuted order: position N1 k2 + k1 holds frequency k2 + N2 k1), times P-hat,
//      inverse N1-point DFT, times w_N^{+m k2}, back in place: forward and inverse of this step
//      touch the same N1 positions, so P-hat is applied between them in registers;
//   3. (line, n1): the N2 points n1 + N1 m, inverse N2-point DFT, times e^{i pi t / N} / N,
//      straight to global memory at t = n1 + N1 m (the 16 lines of one t: 128 contiguous bytes).
// Against separate forward and inverse steps with P-hat between them, the middle step saves two
// passes over the tile and two barriers, and the direct stores a third pass.
template <int N, bool FWD>
__device__ __forceinline__ void tau_outer(float2* __restrict__ sm, float2* __restrict__ y, int64_t inner, float sc,
                                          const float2* tw, const float2* twist) {
    constexpr int N1 = TauSplit<N>::N1, N2 = TauSplit<N>::N2;
    constexpr int total = kTauLines * N1;
#pragma unroll 1
    for (int task = threadIdx.x; task < total; task += kTauThreads) {
        const int line = task % kTauLines, f = task / kTauLines;
        float2 v[N2];
        if constexpr (FWD) {
#pragma unroll
            for (int m = 0; m < N2; ++m) v[m] = sm[(f + N1 * m) * kTauLines + line];
#pragma unroll
            for (int m = 0; m < N2; ++m) {
                const float2 w = twist[f + N1 * m];
                v[m] = make_float2(v[m].x * w.x + v[m].y * w.y, v[m].y * w.x - v[m].x * w.y);
            }
            bfly<N2, -1>(v);
#pragma unroll
            for (int m = 1; m < N2; ++m) {
                const float2 w = tw[f * m];   // f * m < N
                v[m] = make_float2(v[m].x * w.x - v[m].y * w.y, v[m].x * w.y + v[m].y * w.x);
            }
#pragma unroll
            for (int m = 0; m < N2; ++m) sm[(f + N1 * m) * kTauLines + line] = v[m];
        } else {
#pragma unroll
            for (int m = 0; m < N2; ++m) v[m] = sm[(f + N1 * m) * kTauLines + line];
            bfly<N2, +1>(v);
#pragma unroll
            for (int m = 0; m < N2; ++m) {
                const float2 w = twist[f + N1 * m];
                y[(int64_t)(f + N1 * m) * inner + line] =
                    make_float2(sc * (v[m].x * w.x - v[m].y * w.y), sc * (v[m].x * w.y + v[m].y * w.x));
            }
        }
    }
}

// y [nrhs][N][inner] in place; grid nrhs * (inner / 16). A.eitw holds e^{i w_n} in the
// digit-permuted order of the split; A.cosk the cos k table in the order of the x and y
// positions. A.part (optional): per block sum P-hat |y-hat|^2 / N (= <y_in, P y_in> when y_in is
// the unitary (x, y) transform of a vector).
// Resident blocks per SM: six (40 registers) for the short lengths; five (48 registers) from N = 80
// on, where the 16-point DFTs of the middle step would spill at 40.
constexpr int tau_min_blocks(int N) { return N >= 80 ? 5 : 6; }
template <int N>
__global__ void __launch_bounds__(kTauThreads, tau_min_blocks(N)) k_tau(FftcArgs A) {
    constexpr int N1 = TauSplit<N>::N1, N2 = TauSplit<N>::N2;
    __shared__ __align__(16) float2 sm[N * kTauLines];
    __shared__ float2 s_tw[N], s_twist[N], s_ew[N];
    __shared__ float s_base[kTauLines];
    __shared__ double red[kTauThreads / 32];
    const int nib = (int)A.nib;
    const int k = blockIdx.x / nib;
    const int64_t i0 = (int64_t)(blockIdx.x % nib) * kTauLines;
    if (A.cgs && !A.cgs[k].active) return;
    float2* y = A.dst + (int64_t)k * N * A.inner + i0;
    // the tile arrives whole (cp.async, 16 bytes: row t = c / 8, column pair c % 8)
    for (int c = threadIdx.x; c < N * kTauLines / 2; c += kTauThreads)
        cp_async16(sm + 2 * c, y + (int64_t)(c >> 3) * A.inner + 2 * (c & 7));
    cp_async_commit();
    for (int i = threadIdx.x; i < N; i += kTauThreads) {
        s_tw[i] = __ldg(A.tw + i);
        s_twist[i] = __ldg(A.twist + i);
        s_ew[i] = __ldg(A.eitw + i);
    }
    if (threadIdx.x < kTauLines) {
        // P-hat = 1 / |K-hat|^2; the momentum part of K-hat depends only on the line
        const int i = (int)(i0 + threadIdx.x);   // inner index (< 4 L^2)
        const int half = 2 * A.L * A.L;          // inner indices of one band
        const int ab = A.bm ? (i >= half ? 1 : 0) : (i & 3) >> 1;
        const int kk = A.bm ? (i - ab * half) >> 1 : i >> 2;
        s_base[threadIdx.x] = A.c0[ab] + A.chx[ab] * __ldg(A.cosk + kk % A.L) + A.chy[ab] * __ldg(A.cosk + kk / A.L);
    }
    cp_async_wait<0>();
    __syncthreads();
    tau_outer<N, true>(sm, y, A.inner, 0.f, s_tw, s_twist);
    __syncthreads();
    float acc = 0.f;
    {
        const int line = threadIdx.x % kTauLines;
        const float base = s_base[line];
#pragma unroll 1
        for (int task = threadIdx.x; task < kTauLines * N2; task += kTauThreads) {
            const int f = task / kTauLines;
            float2* col = sm + N1 * f * kTauLines + line;
            float2 v[N1];
#pragma unroll
            for (int m = 0; m < N1; ++m) v[m] = col[m * kTauLines];
            bfly<N1, -1>(v);
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                const float2 e = s_ew[N1 * f + m];
                const float re = e.x + base;
                const float ph = 1.0f / (re * re + e.y * e.y);
                acc += ph * (v[m].x * v[m].x + v[m].y * v[m].y);
                v[m] = make_float2(v[m].x * ph, v[m].y * ph);
            }
            bfly<N1, +1>(v);
#pragma unroll
            for (int m = 1; m < N1; ++m) {
                const float2 w = s_tw[f * m];   // f * m < N; conjugated
                v[m] = make_float2(v[m].x * w.x + v[m].y * w.y, v[m].y * w.x - v[m].x * w.y);
            }
#pragma unroll
            for (int m = 0; m < N1; ++m) col[m * kTauLines] = v[m];
        }
    }
    __syncthreads();
    tau_outer<N, false>(sm, y, A.inner, A.scale, s_tw, s_twist);
    if (A.part) {
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0) A.part[blockIdx.x] = tot / N;   // block = k * nib + inner block
    }
}

bool fftc_tau_supported(int n) {
#define HMC_CASE(N) if (n == N) return true;
    HMC_TAU2_SIZES(HMC_CASE)
#undef HMC_CASE
    return false;
}

int fftc_tau_freq(int n, int pos) {
#define HMC_CASE(N) \
    if (n == N) return pos / TauSplit<N>::N1 + TauSplit<N>::N2 * (pos % TauSplit<N>::N1);
    HMC_TAU2_SIZES(HMC_CASE)
#undef HMC_CASE
    return -1;
}

int fftc_precond_tau(hmc_ctx* ctx, const Lat& lat, float2* y, int nrhs, const CgScalars* cgs,
                     const PcTables* pt, const float* cosk, double* part, int* nblk_out, bool band_major) {
    const int n = lat.Nt;
    const FftPlan* pl = get_plan(ctx, n);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan");
    const int NL = lines_rt(n);
    FftcArgs A{};
    A.src = y;
    A.dst = y;
    A.outer = nrhs;
    A.inner = 4 * (int64_t)lat.L * lat.L;
    A.opr = 1;
    A.cgs = cgs;
    A.tw = pl->tw32;
    A.scale = (float)(1.0 / (double)n);
    for (int q = 0; q < 2; ++q) {
        A.c0[q] = (float)(-1.0 - ctx->p.dtau * ctx->p.mu[q]);
        A.chx[q] = (float)(-2.0 * ctx->p.dtau * ctx->p.t_h[q]);
        A.chy[q] = (float)(-2.0 * ctx->p.dtau * ctx->p.t_v[q]);
    }
    A.L = lat.L;
    A.bm = band_major ? 1 : 0;
    A.cosk = cosk;
    A.eitw = pt->eitw32;
    A.twist = pt->twist32;
    if (pt->eitw32_tau && A.inner % kTauLines == 0) {
        A.eitw = pt->eitw32_tau;
        A.dst = y;
        A.nib = A.inner / kTauLines;
        A.part = part;
        if (part) {
            if (A.nib * nrhs > ctx->part_cap / 2) return fail(ctx, HMC_ERR_ARG, "fftc: reduction buffer too small");
            *nblk_out = (int)A.nib;
        }
        const dim3 grid((unsigned)(nrhs * A.nib));
#define HMC_CASE(N)                                                 \
        if (n == N) {                                               \
            k_tau<N><<<grid, kTauThreads, 0, ctx->stream>>>(A);     \
            HMC_LAUNCH(ctx, "k_tau");                               \
            return HMC_OK;                                          \
        }
        HMC_TAU2_SIZES(HMC_CASE)
#undef HMC_CASE
    }
    if (A.inner < NL) return fail(ctx, HMC_ERR_STATE, "fftc: unsupported tile");
    A.nib = (A.inner + NL - 1) / NL;
    A.part = part;
    if (part) {
        if (A.nib * nrhs > ctx->part_cap / 2) return fail(ctx, HMC_ERR_ARG, "fftc: reduction buffer too small");
        *nblk_out = (int)A.nib;
    }
    const dim3 grid((unsigned)(nrhs * A.nib));
#define HMC_CASE(N) \
    if (n == N) return launch_one<N, 0, kTau, -1>(ctx, grid, A);
    HMC_FFTC_SIZES(HMC_CASE)
#undef HMC_CASE
    return fail(ctx, HMC_ERR_STATE, "fftc: unsupported length");
}

// x-axis passes fused with the CG update (forward) or the <r, z> dot (inverse).
int fftc_x_cg(hmc_ctx* ctx, const Lat& lat, int mode, const float2* src, float2* dst, float2* x, float2* r,
              const float2* p, const float2* q, int nrhs, const CgScalars* cgs, double* part, int* nblk_out) {
    const int n = lat.L;
    const FftPlan* pl = get_plan(ctx, n);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan");
    const int OB = lines_rt(n) / 4;
    FftcArgs A{};
    A.src = src;
    A.dst = dst;
    A.x = x;
    A.r = r;
    A.p = p;
    A.q = q;
    A.opr = (int64_t)lat.Nt * lat.L;
    A.outer = A.opr * nrhs;
    A.inner = 4;
    A.nib = 1;
    A.cgs = cgs;
    A.part = part;
    A.tw = pl->tw32;
    A.scale = (float)(1.0 / std::sqrt((double)n));
    const int64_t nblk = (A.opr + OB - 1) / OB;
    if (nblk * nrhs > ctx->part_cap / 2) return fail(ctx, HMC_ERR_ARG, "fftc: reduction buffer too small");
    const dim3 grid((unsigned)nblk, nrhs);
    *nblk_out = (int)nblk;
#define HMC_CASE(N)                                                                     \
    if (n == N) return mode == kXUpd ? launch_one<N, 4, kXUpd, -1>(ctx, grid, A)       \
                                     : launch_one<N, 4, kXDot, +1>(ctx, grid, A);
    HMC_FFTC_SIZES(HMC_CASE)
#undef HMC_CASE
    return fail(ctx, HMC_ERR_STATE, "fftc: unsupported length");
}


// ---- (x, y) passes of the preconditioner inside PCG ------------------------------------------
// One block transforms one band (the two spin components, 16 bytes per site) of one (RHS, tau)
// plane in shared memory along both axes, so the x and y passes cost one read and one write of
// the vector instead of two. Each axis is a two-factor Cooley-Tukey split L = N1 * N2 done in
// place: with n = n1 + N1 n2 and k = k2 + N2 k1,
//   step A (fixed n1): N2-point DFT over n2, times w_L^{n1 k2}, written back to n1 + N1 k2;
//   step B (fixed k2): N1-point DFT over n1 at positions N1 k2 + n1, written back in place.
// Position N1 k2 + k1 then holds frequency k2 + N2 k1: the forward pass leaves the spectrum
// in this digit-permuted order (the tau pass reads its cos k table in the same order) and the
// inverse pass (step B then step A, conjugate twiddles) takes it back to natural order. A task
// transforms one line for both spins (16-byte shared-memory accesses).
template <int L> struct XYSplit { static constexpr int N1 = 0, N2 = 0; };
template <> struct XYSplit<12> { static constexpr int N1 = 4, N2 = 3; };
template <> struct XYSplit<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct XYSplit<20> { static constexpr int N1 = 5, N2 = 4; };
template <> struct XYSplit<24> { static constexpr int N1 = 6, N2 = 4; };
template <> struct XYSplit<40> { static constexpr int N1 = 8, N2 = 5; };
template <> struct XYSplit<80> { static constexpr int N1 = 10, N2 = 8; };
#define HMC_FFTXY_SIZES(X) X(12) X(16) X(20) X(24) X(40) X(80)

constexpr int kXYThreads = 320;
// row stride (in sites) of the shared plane: = 1 mod 8 so that eight consecutive rows at one
// column fall in distinct bank groups
constexpr int xy_row_stride(int L) { return L + ((9 - L % 8) % 8); }
template <int L> constexpr size_t xy_smem_bytes() { return (size_t)L * xy_row_stride(L) * sizeof(float4); }

// In-place DFTs of size R over the positions base(line) + S * m, m < R, for every (line, f)
// task, both spins at once; AX = 0: lines along x (line = row y), AX = 1: lines along y
// (line = column x). STEP_A: f = n1, positions n1 + N1 m; else f = k2, positions N1 k2 + m.
// TW multiplies output m by w_L^{DIR f m} (twiddle table tw in shared memory, forward sign).
template <int L, int AX, bool STEP_A, bool TW, int DIR>
__device__ __forceinline__ void xy_step(float4* sm, const float2* tw) {
    constexpr int N1 = XYSplit<L>::N1, N2 = XYSplit<L>::N2, RS = xy_row_stride(L);
    constexpr int R = STEP_A ? N2 : N1;
    constexpr int NF = STEP_A ? N1 : N2;
    constexpr int total = L * NF;
#pragma unroll 1
    for (int task = threadIdx.x; task < total; task += kXYThreads) {
        const int a = task % L, f = task / L;
        float4* base = AX == 0 ? sm + a * RS + (STEP_A ? f : N1 * f) : sm + a + (STEP_A ? f : N1 * f) * RS;
        constexpr int S = (STEP_A ? N1 : 1) * (AX == 0 ? 1 : RS);   // stride between the R points
        float2 u[R], v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const float4 e = base[m * S];
            u[m] = make_float2(e.x, e.y);
            v[m] = make_float2(e.z, e.w);
        }
        bfly<R, DIR>(u);
        bfly<R, DIR>(v);
        if constexpr (TW) {
#pragma unroll
            for (int m = 1; m < R; ++m) {
                float2 w = tw[f * m];   // f * m < L
                if (DIR > 0) w.y = -w.y;
                u[m] = make_float2(u[m].x * w.x - u[m].y * w.y, u[m].x * w.y + u[m].y * w.x);
                v[m] = make_float2(v[m].x * w.x - v[m].y * w.y, v[m].x * w.y + v[m].y * w.x);
            }
        }
#pragma unroll
        for (int m = 0; m < R; ++m) base[m * S] = make_float4(u[m].x, u[m].y, v[m].x, v[m].y);
    }
}

// dst = F_xy src (DIR -1, permuted order out) or F_xy^-1 src (DIR +1, permuted order in).
// PUPD (DIR +1): dst = F_xy^-1 src + beta_k pold instead, the CG direction update
// p_{k+1} = z + beta_k p_k (A.p = pold, which must not alias dst). Grid (2 Nt, nrhs): block
// (2 t + band, k); right-hand sides with cgs[k].active == 0 are skipped when cgs is given.
// The spectrum (dst of the forward pass, src of the inverse) is band-major, [k][t][band][site]
// [spin]: a block reads or writes its band of the plane as one contiguous run there, where the
// site layout gives it 16 of every 32 bytes (a copy through the block measured 75 us against
// 120 us at 80x80x160 with 8 RHS). dst must not overlap src: the two layouts interleave the
// bands differently, so a block's writes would reach the other band's unread input.
template <int L, int DIR, bool PUPD>
__global__ void __launch_bounds__(kXYThreads, 2) k_fft_xy(FftcArgs A, int Nt) {
    static_assert(!PUPD || DIR > 0, "the direction update follows the inverse pass");
    constexpr int RS = xy_row_stride(L);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 tws[L];
    float4* sm = reinterpret_cast<float4*>(smem_raw);   // [L][RS] sites, both spins
    const int k = blockIdx.y;
    if (A.cgs && !A.cgs[k].active) return;
    const int t = blockIdx.x >> 1, band = blockIdx.x & 1;
    const int64_t g0 = (((int64_t)k * Nt + t) * L * L) * 4 + 2 * band;   // site layout: site 0's band
    const int64_t gz = (((int64_t)k * Nt + t) * 2 + band) * L * L * 2;    // spectrum: the band-plane
    for (int i = threadIdx.x; i < L; i += kXYThreads) tws[i] = __ldg(A.tw + i);

    // the whole band-plane is requested at once (cp.async, 16 bytes per site)
    for (int e = threadIdx.x; e < L * L; e += kXYThreads)
        cp_async16(sm + (e / L) * RS + e % L, A.src + (DIR < 0 ? g0 + 4 * (int64_t)e : gz + 2 * (int64_t)e));
    cp_async_commit();
    if constexpr (PUPD) {
        // pold is read only when the transform is done: bring it into L2 meanwhile (one
        // prefetch per 128-byte line: four sites)
        for (int e = 4 * threadIdx.x; e < L * L; e += 4 * kXYThreads)
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(A.p + g0 + 4 * (int64_t)e));
    }
    cp_async_wait<0>();
    __syncthreads();
    if constexpr (DIR < 0) {
        xy_step<L, 0, true, true, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 0, false, false, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 1, true, true, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 1, false, false, DIR>(sm, tws);
    } else {
        xy_step<L, 1, false, true, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 1, true, false, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 0, false, true, DIR>(sm, tws);
        __syncthreads();
        xy_step<L, 0, true, false, DIR>(sm, tws);
    }
    __syncthreads();
    const float sc = 1.0f / (float)L;   // unitary on both axes
    if constexpr (PUPD) {
        const float beta = (float)A.cgs[k].beta;
        constexpr int XB = 4;   // sites per batch: the batch's loads of pold come before its stores
        for (int e0 = threadIdx.x; e0 < L * L; e0 += XB * kXYThreads) {
            float4 po[XB];
#pragma unroll
            for (int b = 0; b < XB; ++b) {
                const int e = e0 + b * kXYThreads;
                if (e < L * L) po[b] = *reinterpret_cast<const float4*>(A.p + g0 + 4 * (int64_t)e);
            }
#pragma unroll
            for (int b = 0; b < XB; ++b) {
                const int e = e0 + b * kXYThreads;
                if (e < L * L) {
                    const float4 v = sm[(e / L) * RS + e % L];
                    *reinterpret_cast<float4*>(A.dst + g0 + 4 * (int64_t)e) =
                        make_float4(v.x * sc + beta * po[b].x, v.y * sc + beta * po[b].y, v.z * sc + beta * po[b].z,
                                    v.w * sc + beta * po[b].w);
                }
            }
        }
    } else {
        for (int e = threadIdx.x; e < L * L; e += kXYThreads) {
            float4 v = sm[(e / L) * RS + e % L];
            v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
            *reinterpret_cast<float4*>(A.dst + (DIR < 0 ? gz + 2 * (int64_t)e : g0 + 4 * (int64_t)e)) = v;
        }
    }
}

// x += alpha p, r -= alpha q and one partial ||r||^2 per band-plane-sized chunk: grid (2 Nt,
// nrhs), so that the partials line up with those of the inverse (x, y) pass.
__global__ void __launch_bounds__(256) k_xy_cg_update(FftcArgs A, int64_t chunk4) {
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (!A.cgs[k].active) return;
    const float alpha = (float)A.cgs[k].alpha;
    const int64_t o = ((int64_t)k * gridDim.x + blockIdx.x) * chunk4;   // float4 index
    float4* x = reinterpret_cast<float4*>(A.x) + o;
    float4* r = reinterpret_cast<float4*>(A.r) + o;
    const float4* p = reinterpret_cast<const float4*>(A.p) + o;
    const float4* q = reinterpret_cast<const float4*>(A.q) + o;
    float acc = 0.f;
    constexpr int XB = 4;
    for (int64_t e0 = threadIdx.x; e0 < chunk4; e0 += XB * 256) {
        float4 xx[XB], rr[XB], pp[XB], qq[XB];
#pragma unroll
        for (int b = 0; b < XB; ++b) {
            const int64_t e = e0 + b * 256;
            if (e < chunk4) { xx[b] = x[e]; rr[b] = r[e]; pp[b] = p[e]; qq[b] = q[e]; }
        }
#pragma unroll
        for (int b = 0; b < XB; ++b) {
            const int64_t e = e0 + b * 256;
            if (e < chunk4) {
                xx[b].x += alpha * pp[b].x; xx[b].y += alpha * pp[b].y; xx[b].z += alpha * pp[b].z; xx[b].w += alpha * pp[b].w;
                rr[b].x -= alpha * qq[b].x; rr[b].y -= alpha * qq[b].y; rr[b].z -= alpha * qq[b].z; rr[b].w -= alpha * qq[b].w;
                x[e] = xx[b];
                r[e] = rr[b];
                acc += rr[b].x * rr[b].x + rr[b].y * rr[b].y + rr[b].z * rr[b].z + rr[b].w * rr[b].w;
            }
        }
    }
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) A.part[(int64_t)k * gridDim.x + blockIdx.x] = tot;
}

bool fftc_xy_supported(int L) {
#define HMC_CASE(N) if (L == N) return true;
    HMC_FFTXY_SIZES(HMC_CASE)
#undef HMC_CASE
    return false;
}

int fftc_xy_freq(int L, int pos) {
#define HMC_CASE(N) \
    if (L == N) return pos / XYSplit<N>::N1 + XYSplit<N>::N2 * (pos % XYSplit<N>::N1);
    HMC_FFTXY_SIZES(HMC_CASE)
#undef HMC_CASE
    return -1;
}

template <int L, int DIR, bool PUPD>
static int launch_xy(hmc_ctx* ctx, const FftcArgs& A, int Nt, int nrhs) {
    constexpr size_t sm = xy_smem_bytes<L>();
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fft_xy<L, DIR, PUPD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm));
        attr.mark(bit);
    }
    const int64_t n2 = (int64_t)nrhs * Nt * L * L * 4;   // float2 per vector
    if (A.src < A.dst + n2 && A.dst < A.src + n2) return fail(ctx, HMC_ERR_ARG, "fftc: (x, y) pass in place");
    k_fft_xy<L, DIR, PUPD><<<dim3((unsigned)(2 * Nt), nrhs), kXYThreads, sm, ctx->stream>>>(A, Nt);
    HMC_LAUNCH(ctx, "k_fft_xy");
    return HMC_OK;
}

int fftc_xy_update(hmc_ctx* ctx, const Lat& lat, float2* x, float2* r, const float2* p, const float2* q, int nrhs,
                   const CgScalars* cgs, double* part, int* nblk_out) {
    FftcArgs A{};
    A.x = x;
    A.r = r;
    A.p = p;
    A.q = q;
    A.cgs = cgs;
    A.part = part;
    const int64_t nblk = 2 * (int64_t)lat.Nt;
    if (nblk * nrhs > ctx->part_cap / 2) return fail(ctx, HMC_ERR_ARG, "fftc: reduction buffer too small");
    *nblk_out = (int)nblk;
    k_xy_cg_update<<<dim3((unsigned)nblk, nrhs), 256, 0, ctx->stream>>>(A, (int64_t)lat.L * lat.L);
    HMC_LAUNCH(ctx, "k_xy_cg_update");
    return HMC_OK;
}

int fftc_xy_apply(hmc_ctx* ctx, const Lat& lat, const float2* src, float2* dst, int nrhs, int dir,
                  const CgScalars* cgs) {
    const int L = lat.L;
    const FftPlan* pl = get_plan(ctx, L);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan");
    FftcArgs A{};
    A.src = src;
    A.dst = dst;
    A.cgs = cgs;
    A.tw = pl->tw32;
#define HMC_CASE(N)                                                                            \
    if (L == N) return dir < 0 ? launch_xy<N, -1, false>(ctx, A, lat.Nt, nrhs)                  \
                               : launch_xy<N, +1, false>(ctx, A, lat.Nt, nrhs);
    HMC_FFTXY_SIZES(HMC_CASE)
#undef HMC_CASE
    return fail(ctx, HMC_ERR_STATE, "fftc: unsupported length");
}

int fftc_xy_inverse_pupd(hmc_ctx* ctx, const Lat& lat, const float2* zhat, const float2* pold, float2* pnew, int nrhs,
                         const CgScalars* cgs) {
    const int L = lat.L;
    const FftPlan* pl = get_plan(ctx, L);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan");
    if (pold == pnew || !cgs) return fail(ctx, HMC_ERR_ARG, "fftc: bad direction-update buffers");
    FftcArgs A{};
    A.src = zhat;
    A.dst = pnew;
    A.p = pold;
    A.cgs = cgs;
    A.tw = pl->tw32;
#define HMC_CASE(N) \
    if (L == N) return launch_xy<N, +1, true>(ctx, A, lat.Nt, nrhs);
    HMC_FFTXY_SIZES(HMC_CASE)
#undef HMC_CASE
    return fail(ctx, HMC_ERR_STATE, "fftc: unsupported length");
}

}  // namespace hmc
