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

constexpr RadixList radices(int N) {
    RadixList l{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
    while (N % 4 == 0) { l.r[l.n++] = 4; N /= 4; }
    while (N % 2 == 0) { l.r[l.n++] = 2; N /= 2; }
    while (N % 3 == 0) { l.r[l.n++] = 3; N /= 3; }
    while (N % 5 == 0) { l.r[l.n++] = 5; N /= 5; }
    return l;
}

constexpr int kThreads = 256;

template <int R, int DIR>
__device__ __forceinline__ void bfly(float2* v, const float2* __restrict__ tw, int N) {
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
    } else {
        float2 out[R];
        const int step = N / R;
#pragma unroll
        for (int p = 0; p < R; ++p) {
            float2 acc = v[0];
#pragma unroll
            for (int q = 1; q < R; ++q) {
                float2 w = __ldg(tw + ((p * q) % R) * step);
                if (DIR > 0) w.y = -w.y;
                acc.x += v[q].x * w.x - v[q].y * w.y;
                acc.y += v[q].x * w.y + v[q].y * w.x;
            }
            out[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < R; ++p) v[p] = out[p];
    }
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
        bfly<R, DIR>(v, tw, N);
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
        // (both lines share alpha and k: they are spins s = 0, 1 of one site)
        const int64_t i = i0 + icp;
        float base = 0.f;
        if (lane_live) {
            const int ab = (int)((i & 3) >> 1);
            const int kk = (int)(i >> 2);
            const int mx = kk % A.L, my = kk / A.L;
            base = A.c0[ab] + A.chx[ab] * __ldg(A.cosk + mx) + A.chy[ab] * __ldg(A.cosk + my);
        }
#pragma unroll 4
        for (int j = j0; j < N; j += JS) {
            const float2 ew = __ldg(A.eitw + j);
            const float re = ew.x + base;
            const float ph = 1.0f / (re * re + ew.y * ew.y);
            float4 v = *reinterpret_cast<float4*>(res + j * NL + icp);
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
}

// ---- dispatch ------------------------------------------------------------------------------
template <int N> constexpr int lines_for() { return N > 96 ? 16 : 32; }

template <int N, int IC, int MODE, int DIR>
static int launch_one(hmc_ctx* ctx, dim3 grid, const FftcArgs& A) {
    constexpr int NL = lines_for<N>();
    constexpr int ICr = (IC == 4) ? 4 : NL;
    const size_t sm = 2 * (size_t)N * NL * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fftc<N, NL, ICr, MODE, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm));
        attr = true;
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

int fftc_precond_tau(hmc_ctx* ctx, const Lat& lat, float2* y, int nrhs, const CgScalars* cgs,
                     const PcTables* pt) {
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
    A.cosk = pt->cosk32;
    A.eitw = pt->eitw32;
    A.twist = pt->twist32;
    if (A.inner < NL) return fail(ctx, HMC_ERR_STATE, "fftc: unsupported tile");
    A.nib = (A.inner + NL - 1) / NL;
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

}  // namespace hmc
