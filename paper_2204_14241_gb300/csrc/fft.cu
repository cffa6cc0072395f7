// Mixed-radix Stockham FFT along one axis of a strided array, the twisted-Fourier
// preconditioner P = F~ P-hat F~^* (Eqs. twist, Kdiag, precon), and the Fourier-diagonal
// metric operations of Section "Online metric estimation".
//
// A block loads a tile of `nl` lines of length n into shared memory ([j][line] layout, so
// threads working on consecutive lines touch consecutive words), runs every radix stage
// there (Stockham autosort, ping-pong buffers) and writes the tile back. Twiddles come from
// a per-length table e^{-2 pi i t / n} computed on the host in double precision.
#include <cmath>

#include "internal.h"
#include "fft_ct.h"

namespace hmc {

constexpr int kMaxStages = 16;

struct StagePlan {
    int n;
    int nst;
    int radix[kMaxStages];
};

template <typename C, int R>
__device__ __forceinline__ void dft_small(C* v, const C* __restrict__ tw, int n, int dir) {
    if constexpr (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b); v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        C a = v[0], b = v[1], c = v[2], d = v[3];
        C s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
        // multiply s3 by (dir * i): forward (dir = -1) -> -i
        C s3r; s3r.x = -dir * s3.y; s3r.y = dir * s3.x;
        v[0] = cadd(s0, s2); v[2] = csub(s0, s2);
        v[1] = cadd(s1, s3r); v[3] = csub(s1, s3r);
    } else if constexpr (R == 3) {
        // X_{1,2} = v0 - (v1 + v2)/2 +- dir i (sqrt(3)/2) (v1 - v2)
        using T = decltype(v[0].x);
        constexpr T h = (T)0.86602540378443864676;   // sin(2 pi / 3) = sqrt(3) / 2
        const C a = v[0], b = v[1], c = v[2];
        const T tx = b.x + c.x, ty = b.y + c.y;
        const T dx = dir * h * (b.x - c.x), dy = dir * h * (b.y - c.y);
        const T mx = a.x - (T)0.5 * tx, my = a.y - (T)0.5 * ty;
        v[0].x = a.x + tx; v[0].y = a.y + ty;
        v[1].x = mx - dy;  v[1].y = my + dx;
        v[2].x = mx + dy;  v[2].y = my - dx;
    } else if constexpr (R == 5) {
        // pairs (1, 4) and (2, 3): X_{1,4} = m1 +- i n1, X_{2,3} = m2 +- i n2 with
        // m = v0 + c (v_q + v_{5-q}) terms and n = dir s (v_q - v_{5-q}) terms
        using T = decltype(v[0].x);
        constexpr T c1 = (T)0.30901699437494742410;    // cos(2 pi / 5) = (sqrt 5 - 1) / 4
        constexpr T c2 = (T)-0.80901699437494742410;   // cos(4 pi / 5) = -(sqrt 5 + 1) / 4
        constexpr T s1 = (T)0.95105651629515357212;    // sin(2 pi / 5) = sqrt(10 + 2 sqrt 5) / 4
        constexpr T s2 = (T)0.58778525229247312917;    // sin(4 pi / 5) = sqrt(10 - 2 sqrt 5) / 4
        const C v0 = v[0];
        const T a1x = v[1].x + v[4].x, a1y = v[1].y + v[4].y, a2x = v[2].x + v[3].x, a2y = v[2].y + v[3].y;
        const T b1x = v[1].x - v[4].x, b1y = v[1].y - v[4].y, b2x = v[2].x - v[3].x, b2y = v[2].y - v[3].y;
        const T m1x = v0.x + c1 * a1x + c2 * a2x, m1y = v0.y + c1 * a1y + c2 * a2y;
        const T m2x = v0.x + c2 * a1x + c1 * a2x, m2y = v0.y + c2 * a1y + c1 * a2y;
        const T n1x = dir * (s1 * b1x + s2 * b2x), n1y = dir * (s1 * b1y + s2 * b2y);
        const T n2x = dir * (s2 * b1x - s1 * b2x), n2y = dir * (s2 * b1y - s1 * b2y);
        v[0].x = v0.x + a1x + a2x; v[0].y = v0.y + a1y + a2y;
        v[1].x = m1x - n1y; v[1].y = m1y + n1x;
        v[4].x = m1x + n1y; v[4].y = m1y - n1x;
        v[2].x = m2x - n2y; v[2].y = m2y + n2x;
        v[3].x = m2x + n2y; v[3].y = m2y - n2x;
    } else {
        C out[R];
        const int step = n / R;
#pragma unroll
        for (int p = 0; p < R; ++p) {
            C acc = v[0];
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C w = __ldg(tw + ((p * q) % R) * step);
                if (dir > 0) w.y = -w.y;
                acc = cadd(acc, cmul(v[q], w));
            }
            out[p] = acc;
        }
#pragma unroll
        for (int p = 0; p < R; ++p) v[p] = out[p];
    }
}

// One Stockham stage for all lines of the tile: src/dst are [n][nl].
template <typename C, int R>
__device__ __forceinline__ void stage(const C* src, C* dst, int n, int nl, int Ns,
                                      const C* __restrict__ tw, int dir) {
    const int M = n / R;
    const int total = M * nl;
    const int tstep = n / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int line = idx % nl, j = idx / nl;
        const int k = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C a = src[(j + r * M) * nl + line];
            if (r > 0 && k > 0) {
                C w = __ldg(tw + ((r * k * tstep) % n));
                if (dir > 0) w.y = -w.y;
                a = cmul(a, w);
            }
            v[r] = a;
        }
        dft_small<C, R>(v, tw, n, dir);
        const int d = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(d + r * Ns) * nl + line] = v[r];
    }
}

// Runs all stages; returns the buffer holding the result.
template <typename C>
__device__ C* run_stages(C* a, C* b, const StagePlan& sp, int nl, const C* __restrict__ tw, int dir) {
    int Ns = 1;
    for (int s = 0; s < sp.nst; ++s) {
        const int R = sp.radix[s];
        switch (R) {
            case 2: stage<C, 2>(a, b, sp.n, nl, Ns, tw, dir); break;
            case 3: stage<C, 3>(a, b, sp.n, nl, Ns, tw, dir); break;
            case 4: stage<C, 4>(a, b, sp.n, nl, Ns, tw, dir); break;
            case 5: stage<C, 5>(a, b, sp.n, nl, Ns, tw, dir); break;
            default: stage<C, 7>(a, b, sp.n, nl, Ns, tw, dir); break;
        }
        __syncthreads();
        C* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

// Tile geometry: lines are (o, i) with o in [o0, o0 + OB) and i in [i0, i0 + IC).
struct FftTile {
    int64_t outer, inner;
    int OB, IC;
    int64_t nib;   // number of inner blocks
};

template <typename C>
__device__ __forceinline__ void tile_origin(const FftTile& ft, int64_t& o0, int64_t& i0) {
    o0 = (blockIdx.x / ft.nib) * ft.OB;
    i0 = (blockIdx.x % ft.nib) * ft.IC;
}

// out-of-place when src != data (each tile reads src and writes data)
template <typename R>
__global__ void __launch_bounds__(256) k_fft(const cplx<R>* src, cplx<R>* data, FftTile ft, StagePlan sp,
                                             const cplx<R>* __restrict__ tw, int dir, R scale,
                                             const CgScalars* __restrict__ cgs, int64_t opr) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nl = ft.OB * ft.IC, n = sp.n;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + (int64_t)n * nl;
    int64_t o0, i0;
    tile_origin<C>(ft, o0, i0);
    const int tot = n * nl;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int ic = e % ft.IC, rest = e / ft.IC;
        const int j = rest % n, ob = rest / n;
        const int64_t o = o0 + ob, i = i0 + ic;
        if (o < ft.outer && i < ft.inner && !(cgs && !cgs[o / opr].active))
            a[j * nl + ob * ft.IC + ic] = src[(o * n + j) * ft.inner + i];
    }
    __syncthreads();
    C* res = run_stages<C>(a, b, sp, nl, tw, dir);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int ic = e % ft.IC, rest = e / ft.IC;
        const int j = rest % n, ob = rest / n;
        const int64_t o = o0 + ob, i = i0 + ic;
        if (o < ft.outer && i < ft.inner && !(cgs && !cgs[o / opr].active))
            data[(o * n + j) * ft.inner + i] = cscale(res[j * nl + ob * ft.IC + ic], scale);
    }
}

// x-axis FFT passes fused with the CG vector work, one right-hand side per blockIdx.y, data
// [nrhs][Nt * L][L][4]. Lines are (row, component); a tile holds OB whole rows.
//  MODE 1 (forward): x += alpha p, r -= alpha q (written back), partial ||r||^2, then the
//         forward FFT of r along x into out.
//  MODE 2 (inverse): inverse FFT along x of in, written to out, and partial Re<r, out>.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_fft_x_cg(const cplx<R>* in, cplx<R>* out, cplx<R>* __restrict__ xv,
                                                  cplx<R>* __restrict__ rv, const cplx<R>* __restrict__ pv,
                                                  const cplx<R>* __restrict__ qv, int64_t rows, int OB,
                                                  StagePlan sp, const cplx<R>* __restrict__ tw,
                                                  const CgScalars* __restrict__ cgs, double* __restrict__ part) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[8];
    const int k = blockIdx.y;
    if (!cgs[k].active) return;
    const int n = sp.n, nl = OB * 4;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + (int64_t)n * nl;
    const int64_t base = ((int64_t)k * rows + (int64_t)blockIdx.x * OB) * n * 4;   // first element of the tile
    const int64_t nrow = min((int64_t)OB, rows - (int64_t)blockIdx.x * OB);
    const int tot = (int)(nrow * n * 4);
    const R alpha = (R)cgs[k].alpha;
    double acc = 0.0;
    // element e of the tile: row ob = e / (4n), j = (e / 4) % n, component c = e % 4
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int c = e & 3, j = (e >> 2) % n, ob = (e >> 2) / n;
        const int64_t g = base + e;
        C v;
        if constexpr (MODE == 1) {
            C xx = xv[g], r = rv[g];
            const C pp = pv[g], qq = qv[g];
            xx.x += alpha * pp.x; xx.y += alpha * pp.y;
            r.x -= alpha * qq.x; r.y -= alpha * qq.y;
            xv[g] = xx;
            rv[g] = r;
            acc += (double)(r.x * r.x + r.y * r.y);
            v = r;
        } else {
            v = in[g];
        }
        a[j * nl + ob * 4 + c] = v;
    }
    __syncthreads();
    C* res = run_stages<C>(a, b, sp, nl, tw, MODE == 1 ? -1 : +1);
    const R scale = (R)(1.0 / sqrt((double)n));
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int c = e & 3, j = (e >> 2) % n, ob = (e >> 2) / n;
        const int64_t g = base + e;
        const C v = cscale(res[j * nl + ob * 4 + c], scale);
        out[g] = v;
        if constexpr (MODE == 2) {
            const C r = rv[g];
            acc += (double)(r.x * v.x + r.y * v.y);
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[(int64_t)k * gridDim.x + blockIdx.x] = acc;
}

// Preconditioner pass along tau on data [nrhs][Nt][L*L*4] already Fourier transformed in
// x and y: multiply by the twist conj(T) = e^{-i pi t / Nt}, forward FFT over t, multiply by
// P-hat = 1 / |K-hat|^2 with K-hat = e^{i w_n} - 1 - dtau (mu_a + 2 t_h cos kx + 2 t_v cos ky),
// w_n = (2n + 1) pi / Nt, inverse FFT, multiply by T. Inner index i = (m_y * L + m_x) * 4 + c.
struct PrecondCoef {
    double dtau, mu[2], th[2], tv[2];
    int L, Nt;
    const double* cosk;    // cos(2 pi m / L), m < L
    const double2* eitw;   // (cos w_n, sin w_n), n < Nt
    const double2* twist;  // e^{i pi t / Nt}, t < Nt
};

template <typename R>
__global__ void __launch_bounds__(256) k_precond_tau(cplx<R>* __restrict__ data, FftTile ft,
                                                     StagePlan sp, const cplx<R>* __restrict__ tw,
                                                     PrecondCoef pc, R scale2, const CgScalars* __restrict__ cgs) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nl = ft.OB * ft.IC, n = sp.n;
    C* a = reinterpret_cast<C*>(smem_raw);
    C* b = a + (int64_t)n * nl;
    int64_t o0, i0;
    tile_origin<C>(ft, o0, i0);
    const int tot = n * nl;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int ic = e % ft.IC, rest = e / ft.IC;
        const int j = rest % n, ob = rest / n;
        const int64_t o = o0 + ob, i = i0 + ic;
        C v = mk<C>(0.0, 0.0);
        if (o < ft.outer && i < ft.inner && !(cgs && !cgs[o].active)) {
            v = data[(o * n + j) * ft.inner + i];
            const double2 w = pc.twist[j];
            C wc = mk<C>(w.x, -w.y);
            v = cmul(v, wc);
        }
        a[j * nl + ob * ft.IC + ic] = v;
    }
    __syncthreads();
    C* res = run_stages<C>(a, b, sp, nl, tw, -1);
    C* other = (res == a) ? b : a;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int line = e % nl, j = e / nl;
        const int ic = line % ft.IC;
        const int64_t i = i0 + ic;
        if (i < ft.inner) {
            const int c = (int)(i & 3);
            const int alpha = c >> 1;
            const int64_t kk = i >> 2;
            const int mx = (int)(kk % pc.L), my = (int)(kk / pc.L);
            const double eps = 2.0 * pc.th[alpha] * pc.cosk[mx] + 2.0 * pc.tv[alpha] * pc.cosk[my];
            const double2 ew = pc.eitw[j];
            const double re = ew.x - 1.0 - pc.dtau * (pc.mu[alpha] + eps);
            const double im = ew.y;
            const R ph = (R)(1.0 / (re * re + im * im));
            res[j * nl + line] = cscale(res[j * nl + line], ph);
        }
    }
    __syncthreads();
    C* res2 = run_stages<C>(res, other, sp, nl, tw, +1);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int ic = e % ft.IC, rest = e / ft.IC;
        const int j = rest % n, ob = rest / n;
        const int64_t o = o0 + ob, i = i0 + ic;
        if (o < ft.outer && i < ft.inner && !(cgs && !cgs[o].active)) {
            const double2 w = pc.twist[j];
            C v = cmul(res2[j * nl + ob * ft.IC + ic], mk<C>(w.x, w.y));
            data[(o * n + j) * ft.inner + i] = cscale(v, scale2);
        }
    }
}

// ---- host side ----------------------------------------------------------------------------
static std::vector<int> factorize(int n) {
    std::vector<int> f;
    while (n % 4 == 0) { f.push_back(4); n /= 4; }
    while (n % 2 == 0) { f.push_back(2); n /= 2; }
    for (int r : {3, 5, 7})
        while (n % r == 0) { f.push_back(r); n /= r; }
    if (n != 1) f.clear();
    return f;
}

FftPlan* get_plan(hmc_ctx* ctx, int n) {
    for (auto& p : ctx->plans)
        if (p.n == n) return &p;
    return nullptr;
}

static int add_plan(hmc_ctx* ctx, int n) {
    if (get_plan(ctx, n)) return HMC_OK;
    FftPlan p;
    p.n = n;
    p.radix = factorize(n);
    if (p.radix.empty() || (int)p.radix.size() > kMaxStages)
        return fail(ctx, HMC_ERR_ARG, "FFT length " + std::to_string(n) + " must factor into 2, 3, 5, 7");
    std::vector<double2> t64(n);
    std::vector<float2> t32(n);
    for (int k = 0; k < n; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)n;
        t64[k] = make_double2(std::cos(ang), std::sin(ang));
        t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
    }
    HMC_CUDA(ctx, cudaMalloc(&p.tw64, n * sizeof(double2)));
    HMC_CUDA(ctx, cudaMalloc(&p.tw32, n * sizeof(float2)));
    HMC_CUDA(ctx, cudaMemcpy(p.tw64, t64.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(p.tw32, t32.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    ctx->plans.push_back(p);
    return HMC_OK;
}

static PcTables* get_pc(hmc_ctx* ctx, int L, int Nt) {
    for (auto& t : ctx->pcs)
        if (t.L == L && t.Nt == Nt) return &t;
    return nullptr;
}

// Per-lattice preconditioner tables: cos k (L), e^{i w_n} (Nt), twist e^{i pi t / Nt} (Nt).
static int add_pc(hmc_ctx* ctx, int L, int Nt) {
    if (get_pc(ctx, L, Nt)) return HMC_OK;
    PcTables t;
    t.L = L;
    t.Nt = Nt;
    std::vector<double> ck(L);
    std::vector<double2> ew(Nt), tw(Nt);
    for (int m = 0; m < L; ++m) ck[m] = std::cos(2.0 * M_PI * m / L);
    for (int n = 0; n < Nt; ++n) {
        const double w = (2.0 * n + 1.0) * M_PI / Nt;
        ew[n] = make_double2(std::cos(w), std::sin(w));
        const double a = M_PI * n / Nt;
        tw[n] = make_double2(std::cos(a), std::sin(a));
    }
    HMC_CUDA(ctx, cudaMalloc(&t.cosk, L * sizeof(double)));
    HMC_CUDA(ctx, cudaMalloc(&t.eitw, Nt * sizeof(double2)));
    HMC_CUDA(ctx, cudaMalloc(&t.twist, Nt * sizeof(double2)));
    HMC_CUDA(ctx, cudaMemcpy(t.cosk, ck.data(), L * sizeof(double), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(t.eitw, ew.data(), Nt * sizeof(double2), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(t.twist, tw.data(), Nt * sizeof(double2), cudaMemcpyHostToDevice));
    std::vector<float> ck32(L);
    std::vector<float2> ew32(Nt), tw32(Nt);
    for (int m = 0; m < L; ++m) ck32[m] = (float)ck[m];
    for (int n = 0; n < Nt; ++n) {
        ew32[n] = make_float2((float)ew[n].x, (float)ew[n].y);
        tw32[n] = make_float2((float)tw[n].x, (float)tw[n].y);
    }
    HMC_CUDA(ctx, cudaMalloc(&t.cosk32, L * sizeof(float)));
    HMC_CUDA(ctx, cudaMalloc(&t.eitw32, Nt * sizeof(float2)));
    HMC_CUDA(ctx, cudaMalloc(&t.twist32, Nt * sizeof(float2)));
    HMC_CUDA(ctx, cudaMemcpy(t.cosk32, ck32.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(t.eitw32, ew32.data(), Nt * sizeof(float2), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(t.twist32, tw32.data(), Nt * sizeof(float2), cudaMemcpyHostToDevice));
    if (fftc_tau_supported(Nt)) {
        std::vector<float2> ewp(Nt);
        for (int m = 0; m < Nt; ++m) ewp[m] = ew32[fftc_tau_freq(Nt, m)];
        HMC_CUDA(ctx, cudaMalloc(&t.eitw32_tau, Nt * sizeof(float2)));
        HMC_CUDA(ctx, cudaMemcpy(t.eitw32_tau, ewp.data(), Nt * sizeof(float2), cudaMemcpyHostToDevice));
    }
    if (fftc_xy_supported(L)) {
        std::vector<float> ckxy(L);
        for (int m = 0; m < L; ++m) ckxy[m] = (float)std::cos(2.0 * M_PI * fftc_xy_freq(L, m) / L);
        HMC_CUDA(ctx, cudaMalloc(&t.cosk32_xy, L * sizeof(float)));
        HMC_CUDA(ctx, cudaMemcpy(t.cosk32_xy, ckxy.data(), L * sizeof(float), cudaMemcpyHostToDevice));
    }
    ctx->pcs.push_back(t);
    return HMC_OK;
}

int build_plans(hmc_ctx* ctx) {
    for (auto& ch : ctx->chains) {
        int rc;
        if ((rc = add_plan(ctx, ch.lat.L))) return rc;
        if ((rc = add_plan(ctx, ch.lat.Nt))) return rc;
        if ((rc = add_pc(ctx, ch.lat.L, ch.lat.Nt))) return rc;
    }
    return HMC_OK;
}

void free_plans(hmc_ctx* ctx) {
    for (auto& p : ctx->plans) {
        cudaFree(p.tw64);
        cudaFree(p.tw32);
    }
    ctx->plans.clear();
    for (auto& t : ctx->pcs) {
        cudaFree(t.cosk);
        cudaFree(t.eitw);
        cudaFree(t.twist);
        cudaFree(t.cosk32);
        cudaFree(t.eitw32);
        cudaFree(t.twist32);
        cudaFree(t.cosk32_xy);
        cudaFree(t.eitw32_tau);
    }
    ctx->pcs.clear();
}

static StagePlan stage_plan(const FftPlan* p) {
    StagePlan sp;
    sp.n = p->n;
    sp.nst = (int)p->radix.size();
    for (int i = 0; i < sp.nst; ++i) sp.radix[i] = p->radix[i];
    return sp;
}

template <typename R>
static FftTile make_tile(int64_t outer, int n, int64_t inner) {
    FftTile ft;
    ft.outer = outer;
    ft.inner = inner;
    const int target = (sizeof(R) == 8 ? 2048 : 4096) / n;   // lines per tile
    const int want = target < 1 ? 1 : target;
    int cap = (int)(inner < 32 ? inner : 32);
    if (cap > want) cap = want;
    ft.IC = 1;
    while (ft.IC * 2 <= cap) ft.IC *= 2;
    if (inner < 32 && inner <= want) ft.IC = (int)inner;
    int ob = want / ft.IC;
    if (ob < 1) ob = 1;
    if (ob > outer) ob = (int)outer;
    ft.OB = ob;
    ft.nib = (inner + ft.IC - 1) / ft.IC;
    return ft;
}

template <typename R> static const cplx<R>* tw_of(const FftPlan* p);
template <> const float2* tw_of<float>(const FftPlan* p) { return p->tw32; }
template <> const double2* tw_of<double>(const FftPlan* p) { return p->tw64; }

template <typename R>
int fft_axis(hmc_ctx* ctx, cplx<R>* data, int64_t outer, int n, int64_t inner, int dir, const cplx<R>* src,
             const CgScalars* cgs, int64_t opr) {
    if constexpr (sizeof(R) == 4) {
        if (fftc_can(n, inner)) return fftc_axis(ctx, data, outer, n, inner, dir, src, cgs, opr);
    }
    const FftPlan* p = get_plan(ctx, n);
    if (!p) return fail(ctx, HMC_ERR_STATE, "no FFT plan for length " + std::to_string(n));
    FftTile ft = make_tile<R>(outer, n, inner);
    const size_t sm = 2 * (size_t)n * ft.OB * ft.IC * sizeof(cplx<R>);
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fft<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr.mark(bit);
    }
    const int64_t nblk = ((outer + ft.OB - 1) / ft.OB) * ft.nib;
    k_fft<R><<<(unsigned)nblk, 256, sm, ctx->stream>>>(src ? src : data, data, ft, stage_plan(p), tw_of<R>(p), dir,
                                                      (R)(1.0 / std::sqrt((double)n)), cgs, opr > 0 ? opr : 1);
    HMC_LAUNCH(ctx, "k_fft");
    return HMC_OK;
}
template int fft_axis<float>(hmc_ctx*, float2*, int64_t, int, int64_t, int, const float2*, const CgScalars*, int64_t);
template int fft_axis<double>(hmc_ctx*, double2*, int64_t, int, int64_t, int, const double2*, const CgScalars*,
                              int64_t);

// The fused tau pass of the preconditioner on data [nrhs][Nt][L * L * 4] (Fourier space in x, y).
template <typename R>
int precond_tau(hmc_ctx* ctx, const Lat& lat, cplx<R>* y, int nrhs, const CgScalars* cgs) {
    const int L = lat.L, Nt = lat.Nt;
    const FftPlan* p = get_plan(ctx, Nt);
    PcTables* pt = get_pc(ctx, L, Nt);
    if (!p || !pt) return fail(ctx, HMC_ERR_STATE, "no preconditioner plan for this lattice");
    if constexpr (sizeof(R) == 4) {
        if (fftc_can(Nt, 4 * (int64_t)L * L))
            return fftc_precond_tau(ctx, lat, y, nrhs, cgs, pt, pt->cosk32, nullptr, nullptr, false);
    }
    PrecondCoef pc;
    pc.dtau = ctx->p.dtau;
    for (int a = 0; a < 2; ++a) {
        pc.mu[a] = ctx->p.mu[a];
        pc.th[a] = ctx->p.t_h[a];
        pc.tv[a] = ctx->p.t_v[a];
    }
    pc.L = L;
    pc.Nt = Nt;
    pc.cosk = pt->cosk;
    pc.eitw = pt->eitw;
    pc.twist = pt->twist;
    FftTile ft = make_tile<R>(nrhs, Nt, 4 * (int64_t)L * L);
    const size_t sm = 2 * (size_t)Nt * ft.OB * ft.IC * sizeof(cplx<R>);
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_precond_tau<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr.mark(bit);
    }
    const int64_t nblk = ((ft.outer + ft.OB - 1) / ft.OB) * ft.nib;
    k_precond_tau<R><<<(unsigned)nblk, 256, sm, ctx->stream>>>(y, ft, stage_plan(p), tw_of<R>(p), pc,
                                                              (R)(1.0 / (double)Nt), cgs);
    HMC_LAUNCH(ctx, "k_precond_tau");
    return HMC_OK;
}

// y = P x: FFT along x (reading x, writing y), along y, the fused tau pass, inverse y and x.
template <typename R>
int launch_precond(hmc_ctx* ctx, const Lat& lat, const cplx<R>* x, cplx<R>* y, int nrhs, cplx<R>* scratch) {
    const int L = lat.L, Nt = lat.Nt;
    int rc;
    if constexpr (sizeof(R) == 4) {
        // the (x, y) passes and tau pass that PCG runs, with the (band-major) spectrum in scratch:
        // those passes do not run in place
        const PcTables* pt = get_pc(ctx, L, Nt);
        const int64_t n = (int64_t)nrhs * Nt * L * L * 4;
        auto apart = [n](const void* a, const void* b) {
            const cplx<R>* u = static_cast<const cplx<R>*>(a);
            const cplx<R>* v = static_cast<const cplx<R>*>(b);
            return u + n <= v || v + n <= u;
        };
        if (pt && pt->cosk32_xy && fftc_can(Nt, 4 * (int64_t)L * L) && scratch && apart(scratch, x) &&
            apart(scratch, y)) {
            cplx<R>* mid = scratch;
            if ((rc = fftc_xy_apply(ctx, lat, x, mid, nrhs, -1, nullptr))) return rc;
            if ((rc = fftc_precond_tau(ctx, lat, mid, nrhs, nullptr, pt, pt->cosk32_xy, nullptr, nullptr, true)))
                return rc;
            return fftc_xy_apply(ctx, lat, mid, y, nrhs, +1, nullptr);
        }
    }
    if ((rc = fft_axis<R>(ctx, y, (int64_t)nrhs * Nt * L, L, 4, -1, x))) return rc;
    if ((rc = fft_axis<R>(ctx, y, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, -1))) return rc;
    if ((rc = precond_tau<R>(ctx, lat, y, nrhs, nullptr))) return rc;
    if ((rc = fft_axis<R>(ctx, y, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, +1))) return rc;
    if ((rc = fft_axis<R>(ctx, y, (int64_t)nrhs * Nt * L, L, 4, +1))) return rc;
    return HMC_OK;
}
template int launch_precond<float>(hmc_ctx*, const Lat&, const float2*, float2*, int, float2*);
template int launch_precond<double>(hmc_ctx*, const Lat&, const double2*, double2*, int, double2*);

// One preconditioned-CG vector step for every active RHS (see cg.cu): x += alpha p,
// r -= alpha q with partial ||r||^2 into part_r2, z = P r with partial <r, z> into part_rz.
// Both partial arrays hold rows of *nblk_out entries per RHS.
template <typename R>
int launch_cg_update_precond(hmc_ctx* ctx, const Lat& lat, cplx<R>* x, cplx<R>* r, const cplx<R>* p,
                             const cplx<R>* q, cplx<R>* z, int nrhs, const CgScalars* cgs, double* part_r2,
                             double* part_rz, int* nblk_out, int* nblk_rz_out) {
    const int L = lat.L, Nt = lat.Nt;
    const FftPlan* pl = get_plan(ctx, L);
    if (!pl) return fail(ctx, HMC_ERR_STATE, "no FFT plan for length " + std::to_string(L));
    const int64_t rows = (int64_t)Nt * L;
    const int want = (sizeof(R) == 8 ? 2048 : 4096) / L / 4;
    int OB = 1;
    while (OB * 2 <= (want < 1 ? 1 : want)) OB *= 2;
    const int64_t nblk = (rows + OB - 1) / OB;
    if (nblk * nrhs > ctx->part_cap / 2) return fail(ctx, HMC_ERR_ARG, "cg update: reduction buffer too small");
    const size_t sm = 2 * (size_t)L * OB * 4 * sizeof(cplx<R>);
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fft_x_cg<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_fft_x_cg<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        attr.mark(bit);
    }
    int rc;
    if constexpr (sizeof(R) == 4) {
        if (fftc_supported(L)) {
            if ((rc = fftc_x_cg(ctx, lat, kFftcXUpd, nullptr, z, x, r, p, q, nrhs, cgs, part_r2, nblk_out))) return rc;
            if ((rc = fft_axis<R>(ctx, z, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, -1, nullptr, cgs, Nt))) return rc;
            if ((rc = precond_tau<R>(ctx, lat, z, nrhs, cgs))) return rc;
            if ((rc = fft_axis<R>(ctx, z, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, +1, nullptr, cgs, Nt))) return rc;
            if ((rc = fftc_x_cg(ctx, lat, kFftcXDot, z, z, nullptr, r, nullptr, nullptr, nrhs, cgs, part_rz,
                                nblk_rz_out)))
                return rc;
            return HMC_OK;
        }
    }
    const dim3 grid((unsigned)nblk, nrhs);
    const StagePlan sp = stage_plan(pl);
    k_fft_x_cg<R, 1><<<grid, 256, sm, ctx->stream>>>(nullptr, z, x, r, p, q, rows, OB, sp, tw_of<R>(pl), cgs, part_r2);
    HMC_LAUNCH(ctx, "k_fft_x_cg<1>");
    if ((rc = fft_axis<R>(ctx, z, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, -1, nullptr, cgs, Nt))) return rc;
    if ((rc = precond_tau<R>(ctx, lat, z, nrhs, cgs))) return rc;
    if ((rc = fft_axis<R>(ctx, z, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, +1, nullptr, cgs, Nt))) return rc;
    k_fft_x_cg<R, 2><<<grid, 256, sm, ctx->stream>>>(z, z, nullptr, r, nullptr, nullptr, rows, OB, sp, tw_of<R>(pl), cgs,
                                                      part_rz);
    HMC_LAUNCH(ctx, "k_fft_x_cg<2>");
    *nblk_out = (int)nblk;
    *nblk_rz_out = (int)nblk;
    return HMC_OK;
}
bool pcg_xy_path(hmc_ctx* ctx, const Lat& lat) {
    const PcTables* pt = get_pc(ctx, lat.L, lat.Nt);
    return pt && pt->cosk32_xy && fftc_can(lat.Nt, 4 * (int64_t)lat.L * lat.L);
}

int launch_pcg_xy_forward(hmc_ctx* ctx, const Lat& lat, float2* x, float2* r, const float2* p, const float2* q,
                          float2* zhat, int nrhs, const CgScalars* cgs, double* part_r2, double* part_rz,
                          int* nblk_r2, int* nblk_rz) {
    const PcTables* pt = get_pc(ctx, lat.L, lat.Nt);
    if (!pt || !pt->cosk32_xy) return fail(ctx, HMC_ERR_STATE, "no (x, y) pass for this lattice");
    int rc;
    // the vector update streams on its own; the (x, y) pass leaves the spectrum in digit-permuted
    // order, and the tau pass forms <r, z> = sum P-hat |F~^* r|^2 (F~ unitary) as it applies P-hat
    if ((rc = fftc_xy_update(ctx, lat, x, r, p, q, nrhs, cgs, part_r2, nblk_r2))) return rc;
    if ((rc = fftc_xy_apply(ctx, lat, r, zhat, nrhs, -1, cgs))) return rc;
    return fftc_precond_tau(ctx, lat, zhat, nrhs, cgs, pt, pt->cosk32_xy, part_rz, nblk_rz, true);
}

int launch_pcg_xy_inverse(hmc_ctx* ctx, const Lat& lat, const float2* zhat, const float2* pold, float2* pnew,
                          int nrhs, const CgScalars* cgs) {
    return fftc_xy_inverse_pupd(ctx, lat, zhat, pold, pnew, nrhs, cgs);
}

template int launch_cg_update_precond<float>(hmc_ctx*, const Lat&, float2*, float2*, const float2*, const float2*,
                                             float2*, int, const CgScalars*, double*, double*, int*, int*);
template int launch_cg_update_precond<double>(hmc_ctx*, const Lat&, double2*, double2*, const double2*,
                                              const double2*, double2*, int, const CgScalars*, double*, double*, int*,
                                              int*);

// ---- randomized diagonal estimator of the fermion Green's function ------------------------------
// y[k][t][.] *= e^{sign i pi t / Nt}
__global__ void k_twist(double2* __restrict__ y, const double2* __restrict__ tw, int Nt, int64_t slice, int64_t n,
                        int sign) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = (int)((i / slice) % Nt);
    const double2 w = tw[t];
    const double2 a = y[i];
    const double s = (double)sign;
    y[i] = make_double2(a.x * w.x - s * a.y * w.y, a.y * w.x + s * a.x * w.y);
}

// out[i] = (1/K) sum_k v_k[i] * o_k[i]
__global__ void k_probe_mean(const double2* __restrict__ v, const double2* __restrict__ o, double2* __restrict__ out,
                             int64_t n, int K) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < K; ++k) {
        const double2 a = v[(int64_t)k * n + i], b = o[(int64_t)k * n + i];
        re += a.x * b.x - a.y * b.y;
        im += a.x * b.y + a.y * b.x;
    }
    out[i] = make_double2(re / K, im / K);
}

// F~ (inverse = 1: T times the inverse unitary DFT) or F~^* (inverse = 0: forward DFT of T^* x),
// from src into dst, over (tau, y, x) of each of the nrhs vectors [V][4].
static int twisted_fourier(hmc_ctx* ctx, const Lat& lat, const double2* src, double2* dst, int nrhs, int inverse) {
    const int L = lat.L, Nt = lat.Nt;
    const PcTables* pt = get_pc(ctx, L, Nt);
    if (!pt) return fail(ctx, HMC_ERR_STATE, "no twist table for this lattice");
    const int64_t n = 4 * lat.V * (int64_t)nrhs, slice = 4 * (int64_t)L * L;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const int dir = inverse ? +1 : -1;
    int rc;
    if (!inverse) {
        if (src != dst) HMC_CUDA(ctx, cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
        k_twist<<<nb, 256, 0, ctx->stream>>>(dst, pt->twist, Nt, slice, n, -1);
        HMC_LAUNCH(ctx, "k_twist");
        src = dst;
    }
    if ((rc = fft_axis<double>(ctx, dst, (int64_t)nrhs * Nt * L, L, 4, dir, src))) return rc;
    if ((rc = fft_axis<double>(ctx, dst, (int64_t)nrhs * Nt, L, 4 * (int64_t)L, dir))) return rc;
    if ((rc = fft_axis<double>(ctx, dst, nrhs, Nt, slice, dir))) return rc;
    if (inverse) {
        k_twist<<<nb, 256, 0, ctx->stream>>>(dst, pt->twist, Nt, slice, n, +1);
        HMC_LAUNCH(ctx, "k_twist");
    }
    return HMC_OK;
}

int green_run(hmc_ctx* ctx, int chain, const double* phi, const double2* v, int nrhs, double2* out, int precond,
              hmc_cg_stats* st) {
    const Lat& lat = ctx->chains[chain].lat;
    int rc;
    if ((rc = twisted_fourier(ctx, lat, v, ctx->d_pf, nrhs, 1))) return rc;                        // w = F~ v
    if ((rc = cg_run(ctx, chain, phi, ctx->d_pf, ctx->d_X, nrhs, ctx->p.cg_tol, ctx->p.cg_maxit, precond, st)))
        return rc;                                                                                   // u = A^-1 w
    if ((rc = launch_apply_D<double>(ctx, lat, phi, ctx->d_X, ctx->d_chi, 1, nrhs))) return rc;    // D^dag u
    if ((rc = twisted_fourier(ctx, lat, ctx->d_chi, ctx->d_chi, nrhs, 0))) return rc;              // F~^* D^-1 F~ v
    const int64_t n = 4 * lat.V;
    k_probe_mean<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(v, ctx->d_chi, out, n, nrhs);
    HMC_LAUNCH(ctx, "k_probe_mean");
    return HMC_OK;
}

// ---- metric -----------------------------------------------------------------------------
__global__ void k_pack_real(const double* __restrict__ in, double2* __restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i], 0.0);
}

// mode 0: v *= sig; 1: v /= sqrt(sig); 2: partial sums of 0.5 sig |v|^2; 3: acc += |v|^2;
// 4: partial sums of |v|^2 / sig
__global__ void __launch_bounds__(256) k_spectral(double2* __restrict__ v, const double* __restrict__ sig,
                                                  int64_t n, int mode, double* __restrict__ acc,
                                                  double* __restrict__ part) {
    __shared__ double red[8];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < n) {
        double2 a = v[i];
        if (mode == 0) {
            const double s = sig[i];
            v[i] = make_double2(a.x * s, a.y * s);
        } else if (mode == 1) {
            const double s = 1.0 / sqrt(sig[i]);
            v[i] = make_double2(a.x * s, a.y * s);
        } else if (mode == 2) {
            e = 0.5 * sig[i] * (a.x * a.x + a.y * a.y);
        } else if (mode == 4) {
            e = (a.x * a.x + a.y * a.y) / sig[i];
        } else {
            acc[i] += a.x * a.x + a.y * a.y;
        }
    }
    if (mode == 2 || mode == 4) {
        const double t = block_sum(e, red);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// out = Re(v) (eps == 0) or out += eps Re(v)
__global__ void k_unpack_real(const double2* __restrict__ v, double* __restrict__ out, int64_t n, double eps) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = eps == 0.0 ? v[i].x : out[i] + eps * v[i].x;
}

static int fft3_real_field(hmc_ctx* ctx, const Lat& lat, double2* v, int dir) {
    const int L = lat.L, Nt = lat.Nt;
    int rc;
    if ((rc = fft_axis<double>(ctx, v, 3 * (int64_t)Nt * L, L, 1, dir))) return rc;
    if ((rc = fft_axis<double>(ctx, v, 3 * (int64_t)Nt, L, L, dir))) return rc;
    if ((rc = fft_axis<double>(ctx, v, 3, Nt, (int64_t)L * L, dir))) return rc;
    return HMC_OK;
}

int metric_op(hmc_ctx* ctx, const Lat& lat, int op, const double* sig, const double* in,
              double* out, double eps, double* scalar_dev) {
    const int64_t n = 3 * lat.V;
    const unsigned nb = (unsigned)((n + 255) / 256);
    double2* v = ctx->d_fft;
    k_pack_real<<<nb, 256, 0, ctx->stream>>>(in, v, n);
    HMC_LAUNCH(ctx, "k_pack_real");
    int rc;
    if ((rc = fft3_real_field(ctx, lat, v, -1))) return rc;
    if (op == HMC_METRIC_KINETIC || op == HMC_METRIC_MNORM) {
        if (nb > ctx->part_cap) return fail(ctx, HMC_ERR_ARG, "metric: reduction buffer too small");
        k_spectral<<<nb, 256, 0, ctx->stream>>>(v, sig, n, op == HMC_METRIC_KINETIC ? 2 : 4, nullptr, ctx->d_part);
        HMC_LAUNCH(ctx, "k_spectral");
        return reduce_rows(ctx, ctx->d_part, 1, (int)nb, scalar_dev);
    }
    if (op == HMC_METRIC_ACCUM) {
        k_spectral<<<nb, 256, 0, ctx->stream>>>(v, sig, n, 3, out, nullptr);
        HMC_LAUNCH(ctx, "k_spectral");
        return HMC_OK;
    }
    k_spectral<<<nb, 256, 0, ctx->stream>>>(v, sig, n, op == HMC_METRIC_MOMENTUM ? 1 : 0, nullptr, nullptr);
    HMC_LAUNCH(ctx, "k_spectral");
    if ((rc = fft3_real_field(ctx, lat, v, +1))) return rc;
    k_unpack_real<<<nb, 256, 0, ctx->stream>>>(v, out, n, eps);
    HMC_LAUNCH(ctx, "k_unpack_real");
    return HMC_OK;
}

// ---- deterministic reductions ----------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce_rows(const double* __restrict__ part, int nblk,
                                                     double* __restrict__ out) {
    __shared__ double red[8];
    const double* row = part + (int64_t)blockIdx.x * nblk;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += row[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

int reduce_rows(hmc_ctx* ctx, const double* part, int k, int nblk, double* out) {
    k_reduce_rows<<<k, 256, 0, ctx->stream>>>(part, nblk, out);
    HMC_LAUNCH(ctx, "k_reduce_rows");
    return HMC_OK;
}

}  // namespace hmc
