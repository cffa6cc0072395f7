// Fermion-matrix stencils (Eq. D_formula), the fused normal operator A = D D^dagger
// (Eq. linsys), and the fused force kernel (Eq. hamiltonseq with S = S_B + S_PF).
#include <mutex>

#include "internal.h"

namespace hmc {

template <typename R> Coef<R> make_coef(const hmc_params& p) {
    Coef<R> c;
    for (int a = 0; a < 2; ++a) {
        c.diag[a] = (R)(-1.0 - p.dtau * p.mu[a]);
        c.hx[a] = (R)(-p.dtau * p.t_h[a]);
        c.hy[a] = (R)(-p.dtau * p.t_v[a]);
    }
    c.cpl = (R)(p.dtau * p.g);
    return c;
}
template Coef<float> make_coef<float>(const hmc_params&);
template Coef<double> make_coef<double>(const hmc_params&);

// ---------------------------------------------------------------------------------------
// y = D x or D^dagger x, one thread per site, neighbours through the read-only cache.
template <typename R, bool DAG>
__global__ void __launch_bounds__(256) k_apply_D(Lat lat, Coef<R> cf, const R* __restrict__ phi,
                                                 const Site<R>* __restrict__ x,
                                                 Site<R>* __restrict__ y, const CgScalars* __restrict__ cgs) {
    if (cgs && !cgs[blockIdx.y].active) return;
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= lat.V) return;
    const int64_t V = lat.V;
    const int L = lat.L;
    const Site<R>* xk = x + blockIdx.y * V;
    const int xx = (int)(s % L);
    const int64_t rest = s / L;
    const int yy = (int)(rest % L);
    const int t = (int)(rest / L);
    const int64_t row = s - xx, slice = (int64_t)t * L * L;
    const int tn = DAG ? tprev(t, lat.Nt) : tnext(t, lat.Nt);
    const R tsign = DAG ? (t == 0 ? R(-1) : R(1)) : (t == lat.Nt - 1 ? R(-1) : R(1));
    const R eta = ((xx + yy) & 1) ? R(-1) : R(1);
    auto ld = [&](int64_t i) {
        Site<R> z{};
        return HMC_IN(i >= 0 && i < V, kBndApplyD) ? load_site(xk + i) : z;
    };
    Site<R> o = site_op<R>(cf, ld(s), ld(row + wrap_dec(xx, L)), ld(row + wrap_inc(xx, L)),
                           ld(slice + (int64_t)wrap_dec(yy, L) * L + xx), ld(slice + (int64_t)wrap_inc(yy, L) * L + xx),
                           ld((int64_t)tn * L * L + (s - slice)), tsign,
                           __ldg(phi + s), __ldg(phi + V + s), __ldg(phi + 2 * V + s), eta);
    store_site(y + blockIdx.y * V + s, o);
}

template <typename R>
int launch_apply_D(hmc_ctx* ctx, const Lat& lat, const R* phi, const cplx<R>* x, cplx<R>* y,
                   int dagger, int nrhs, const CgScalars* cgs) {
    if (nrhs <= 0) return HMC_OK;
    dim3 grid((unsigned)((lat.V + 255) / 256), nrhs);
    Coef<R> cf = make_coef<R>(ctx->p);
    auto xs = reinterpret_cast<const Site<R>*>(x);
    auto ys = reinterpret_cast<Site<R>*>(y);
    if (dagger) k_apply_D<R, true><<<grid, 256, 0, ctx->stream>>>(lat, cf, phi, xs, ys, cgs);
    else        k_apply_D<R, false><<<grid, 256, 0, ctx->stream>>>(lat, cf, phi, xs, ys, cgs);
    HMC_LAUNCH(ctx, "k_apply_D");
    return HMC_OK;
}
template int launch_apply_D<float>(hmc_ctx*, const Lat&, const float*, const float2*, float2*, int, int,
                                   const CgScalars*);
template int launch_apply_D<double>(hmc_ctx*, const Lat&, const double*, const double2*, double2*, int, int,
                                    const CgScalars*);

// The FP64 true residual r = b - D t of a reliable update or of a start from a guess, in the
// operator's second pass: the pass is bound by the FP64 pipe, so streaming b in and r (and its
// complex64 copy) out costs no extra time, and the separate residual pass is not needed.
__global__ void __launch_bounds__(256) k_residual_D(Lat lat, Coef<double> cf, const double* __restrict__ phi,
                                                    const Site<double>* __restrict__ t,
                                                    const Site<double>* __restrict__ b, Site<double>* __restrict__ r,
                                                    Site<float>* __restrict__ r32, double* __restrict__ part,
                                                    const CgScalars* __restrict__ cgs) {
    __shared__ double red[8];
    if (cgs && !cgs[blockIdx.y].active) return;
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t V = lat.V;
    double e = 0.0;
    if (s < V) {
        const int L = lat.L;
        const Site<double>* tk = t + blockIdx.y * V;
        const int xx = (int)(s % L);
        const int64_t rest = s / L;
        const int yy = (int)(rest % L);
        const int tt = (int)(rest / L);
        const int64_t row = s - xx, slice = (int64_t)tt * L * L;
        const int tn = tnext(tt, lat.Nt);
        const double tsign = tt == lat.Nt - 1 ? -1.0 : 1.0;
        const double eta = ((xx + yy) & 1) ? -1.0 : 1.0;
        auto ld = [&](int64_t i) {
            Site<double> z{};
            return HMC_IN(i >= 0 && i < V, kBndApplyD) ? load_site(tk + i) : z;
        };
        const Site<double> o = site_op<double>(cf, ld(s), ld(row + wrap_dec(xx, L)), ld(row + wrap_inc(xx, L)),
                                               ld(slice + (int64_t)wrap_dec(yy, L) * L + xx),
                                               ld(slice + (int64_t)wrap_inc(yy, L) * L + xx),
                                               ld((int64_t)tn * L * L + (s - slice)), tsign, __ldg(phi + s),
                                               __ldg(phi + V + s), __ldg(phi + 2 * V + s), eta);
        const int64_t g = blockIdx.y * V + s;
        const Site<double> bb = load_site(b + g);
        Site<double> rr;
        Site<float> rf;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            rr.c[q] = make_double2(bb.c[q].x - o.c[q].x, bb.c[q].y - o.c[q].y);
            rf.c[q] = make_float2((float)rr.c[q].x, (float)rr.c[q].y);
            e += rr.c[q].x * rr.c[q].x + rr.c[q].y * rr.c[q].y;
        }
        store_site(r + g, rr);
        if (r32) store_site(r32 + g, rf);
    }
    e = block_sum(e, red);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = e;
}

int launch_residual_D(hmc_ctx* ctx, const Lat& lat, const double* phi, const double2* t, const double2* b,
                      double2* r64, float2* r32, int nrhs, double* part, int* nblk_out, const CgScalars* cgs) {
    const int nblk = (int)((lat.V + 255) / 256);
    if ((int64_t)nblk * nrhs > ctx->part_cap) return fail(ctx, HMC_ERR_ARG, "residual: reduction buffer too small");
    k_residual_D<<<dim3((unsigned)nblk, nrhs), 256, 0, ctx->stream>>>(
        lat, make_coef<double>(ctx->p), phi, reinterpret_cast<const Site<double>*>(t),
        reinterpret_cast<const Site<double>*>(b), reinterpret_cast<Site<double>*>(r64),
        reinterpret_cast<Site<float>*>(r32), part, cgs);
    HMC_LAUNCH(ctx, "k_residual_D");
    *nblk_out = nblk;
    return HMC_OK;
}

// ---------------------------------------------------------------------------------------
// Fused y = D (D^dagger x). A block owns a TX x TY tile of sites and marches through a
// chunk of time slices. For output slice t it needs t_ = D^dagger x on the tile plus a
// one-site ring at slice t and on the tile at slice t+1; t_ at slice t+1 in turn needs x at
// t+1 on a two-site ring and x at t on the one-site ring. Each step stores x(t+1) (held in
// registers) into shared memory, issues the global loads of x(t+2) into registers so that
// they are in flight while it computes t_(t+1) on the ring and y(t) on the tile. x and t_
// are double buffered in shared memory, phi triple buffered. Shared memory holds each site
// as 16-byte planes (conflict-free vector access).
template <typename R> struct Planes {
    static constexpr int NP = sizeof(Site<R>) / 16;   // 2 for float, 4 for double
};

template <typename R>
__device__ __forceinline__ void sm_store(uint4* base, int n, int i, const Site<R>& s) {
    const uint4* v = reinterpret_cast<const uint4*>(&s);
#pragma unroll
    for (int q = 0; q < Planes<R>::NP; ++q) base[q * n + i] = v[q];
}
template <typename R>
__device__ __forceinline__ Site<R> sm_load(const uint4* base, int n, int i) {
    Site<R> s;
    uint4* v = reinterpret_cast<uint4*>(&s);
#pragma unroll
    for (int q = 0; q < Planes<R>::NP; ++q) v[q] = base[q * n + i];
    return s;
}

struct ATile {
    int TX, TY, C;        // tile extent and time-chunk length
    int ntx, nty, nchunk; // tiles along x, y and chunks along t
};

constexpr int kAThreads = 256;
template <typename R> struct APf { static constexpr int N = sizeof(R) == 4 ? 2 : 1; };  // halo sites per thread

// With pnew != nullptr the kernel also performs the CG direction update: the operand is
// p = x + beta_k * pold (x holding z), formed as it is loaded, and the block writes p for the
// sites it owns (tile interior, slices [t0, t1)) to pnew; y = A p. pold and pnew must differ.
// PUPD: the direction-update variant used inside PCG (pnew, pold non-null); otherwise the
// plain operator. The plain variant carries no second prefetch register set.
template <typename R, bool PUPD>
__global__ void __launch_bounds__(kAThreads, 2)
k_apply_A(Lat lat, Coef<R> cf, ATile tl, const R* __restrict__ phi, const Site<R>* __restrict__ x,
          Site<R>* __restrict__ y, double* __restrict__ part, const CgScalars* __restrict__ cgs,
          const Site<R>* __restrict__ pold, Site<R>* __restrict__ pnew) {
    if (cgs && !cgs[blockIdx.z].active) return;
    constexpr int NPF = APf<R>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = tl.TX, TY = tl.TY;
    const int HX2 = TX + 4, HY2 = TY + 4, N2 = HX2 * HY2;
    const int HX1 = TX + 2, HY1 = TY + 2, N1 = HX1 * HY1;
    uint4* xa = reinterpret_cast<uint4*>(smem_raw);
    uint4* xb = xa + Planes<R>::NP * N2;
    uint4* ta = xb + Planes<R>::NP * N2;
    uint4* tb = ta + Planes<R>::NP * N1;
    R* phb = reinterpret_cast<R*>(tb + Planes<R>::NP * N1);   // 3 buffers of [3][N1]
    __shared__ double red[kAThreads / 32];

    const int L = lat.L, Nt = lat.Nt;
    const int64_t V = lat.V, LL = (int64_t)L * L;
    const int tile = blockIdx.x;
    const int x0 = (tile % tl.ntx) * TX, y0 = (tile / tl.ntx) * TY;
    const int t0 = blockIdx.y * tl.C;
    const int t1 = min(t0 + tl.C, Nt);
    const int k = blockIdx.z;
    const Site<R>* xk = x + k * V;
    Site<R>* yk = y + k * V;
    const R beta = PUPD ? (R)cgs[k].beta : R(0);
    const Site<R>* pok = PUPD ? pold + k * V : nullptr;
    Site<R>* pnk = PUPD ? pnew + k * V : nullptr;

    auto gx = [&](int i) { int v = (x0 + i) % L; return v < 0 ? v + L : v; };
    auto gy = [&](int j) { int v = (y0 + j) % L; return v < 0 ? v + L : v; };

    // Per-thread geometry, fixed for the whole march: in-plane offsets (y * L + x) of this
    // thread's two-site-ring sites (x loads), one-site-ring sites (phi loads and t_ outputs)
    // and of its tile site (y output). -1 marks "none".
    int h2o[NPF], h1o[NPF], mtc[NPF];
    bool h2own[NPF], h2ring[NPF];
    R mte[NPF];
#pragma unroll
    for (int j = 0; j < NPF; ++j) {
        const int i = threadIdx.x + j * kAThreads;
        h2o[j] = -1; h1o[j] = -1; mtc[j] = 0; h2own[j] = false; h2ring[j] = false; mte[j] = R(1);
        if (i < N2) {
            const int hx = i % HX2, hy = i / HX2;
            h2o[j] = gy(hy - 2) * L + gx(hx - 2);
            h2own[j] = hx >= 2 && hy >= 2 && hx < TX + 2 && hy < TY + 2 && x0 + hx - 2 < L && y0 + hy - 2 < L;
            h2ring[j] = hx == 0 || hy == 0 || hx == HX2 - 1 || hy == HY2 - 1;
        }
        if (i < N1) {
            const int hx = i % HX1, hy = i / HX1;
            const int X = gx(hx - 1), Y = gy(hy - 1);
            h1o[j] = Y * L + X;
            mtc[j] = (hy + 1) * HX2 + hx + 1;
            mte[j] = ((X + Y) & 1) ? R(-1) : R(1);
        }
    }
    int yo = -1, yc = 0;
    R ye = R(1);
    if (threadIdx.x < TX * TY) {
        const int ix = threadIdx.x % TX, iy = threadIdx.x / TX;
        const int X = x0 + ix, Y = y0 + iy;
        if (X < L && Y < L) {
            yo = Y * L + X;
            yc = (iy + 1) * HX1 + ix + 1;
            ye = ((X + Y) & 1) ? R(-1) : R(1);
        }
    }

    // register prefetch of one slice: x on this thread's two-site-ring sites, phi on its
    // one-site-ring sites
    Site<R> rz[NPF];
    Site<R> rp[PUPD ? NPF : 1];
    R rph[NPF][3];
    auto fetch = [&](int t) {
        const int64_t base = (int64_t)t * LL;
#pragma unroll
        for (int j = 0; j < NPF; ++j) {
            if (h2o[j] >= 0) {
                rz[j] = load_site(xk + base + h2o[j]);
                if constexpr (PUPD) rp[j] = load_site(pok + base + h2o[j]);
            }
            if (h1o[j] >= 0) {
                const R* pp = phi + base + h1o[j];
                rph[j][0] = __ldg(pp);
                rph[j][1] = __ldg(pp + V);
                rph[j][2] = __ldg(pp + 2 * V);
            }
        }
    };
    // store the prefetched slice t (p = z + beta pold, written to pnew where owned)
    auto commit = [&](uint4* dst, R* ph, int t, bool own, bool ring1only) {
        const int64_t base = (int64_t)t * LL;
#pragma unroll
        for (int j = 0; j < NPF; ++j) {
            const int i = threadIdx.x + j * kAThreads;
            if (h2o[j] >= 0 && !(ring1only && h2ring[j])) {
                Site<R> v = rz[j];
                if constexpr (PUPD) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v.c[q].x += beta * rp[j].c[q].x;
                        v.c[q].y += beta * rp[j].c[q].y;
                    }
                    if (own && h2own[j]) store_site(pnk + base + h2o[j], v);
                }
                sm_store<R>(dst, N2, i, v);
            }
            if (h1o[j] >= 0 && ph) {
                ph[i] = rph[j][0];
                ph[N1 + i] = rph[j][1];
                ph[2 * N1 + i] = rph[j][2];
            }
        }
    };
    // t_(t) = D^dagger x on the one-site ring from x(t) (cur) and x(t-1) (prev)
    auto make_t = [&](uint4* dst, const uint4* cur, const uint4* prev, const R* ph, int t) {
        const R tsign = (t == 0) ? R(-1) : R(1);   // b(t-1)
#pragma unroll
        for (int j = 0; j < NPF; ++j) {
            if (h1o[j] < 0) continue;
            const int i = threadIdx.x + j * kAThreads;
            const int c = mtc[j];
            Site<R> o = site_op<R>(cf, sm_load<R>(cur, N2, c), sm_load<R>(cur, N2, c - 1),
                                   sm_load<R>(cur, N2, c + 1), sm_load<R>(cur, N2, c - HX2),
                                   sm_load<R>(cur, N2, c + HX2), sm_load<R>(prev, N2, c), tsign,
                                   ph[i], ph[N1 + i], ph[2 * N1 + i], mte[j]);
            sm_store<R>(dst, N1, i, o);
        }
    };

    // prologue: x(t0) on the two-site ring, x(t0 - 1) on the one-site ring, t_(t0)
    fetch(t0);
    commit(xa, phb, t0, true, false);
    fetch(tprev(t0, Nt));
    commit(xb, nullptr, tprev(t0, Nt), false, true);
    __syncthreads();
    make_t(ta, xa, xb, phb, t0);
    fetch(tnext(t0, Nt));
    __syncthreads();

    uint4 *xc = xa, *xn = xb, *tc = ta, *tn = tb;
    int pc = 0;   // phi(t) is in buffer pc of the three at phb
    R acc = 0;   // per-thread partial in the operator's precision
    for (int t = t0; t < t1; ++t) {
        const int tp = tnext(t, Nt);
        const int pn = pc == 2 ? 0 : pc + 1;
        R* phn = phb + pn * 3 * N1;
        commit(xn, phn, tp, t + 1 < t1, false);
        if (t + 1 < t1) fetch(tnext(tp, Nt));
        __syncthreads();
        make_t(tn, xn, xc, phn, tp);
        __syncthreads();
        // y(t) = D t_ on the tile
        if (yo >= 0) {
            const R tsign = (t == Nt - 1) ? R(-1) : R(1);   // b(t)
            const R* ph = phb + pc * 3 * N1;
            const int c = yc;
            const Site<R> tcen = sm_load<R>(tc, N1, c);
            Site<R> o = site_op<R>(cf, tcen, sm_load<R>(tc, N1, c - 1), sm_load<R>(tc, N1, c + 1),
                                   sm_load<R>(tc, N1, c - HX1), sm_load<R>(tc, N1, c + HX1),
                                   sm_load<R>(tn, N1, c), tsign, ph[c], ph[N1 + c], ph[2 * N1 + c], ye);
            store_site(yk + (int64_t)t * LL + yo, o);
            if (part) {
                R n2 = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) n2 += tcen.c[q].x * tcen.c[q].x + tcen.c[q].y * tcen.c[q].y;
                acc += n2;
            }
        }
        uint4* sw = xc; xc = xn; xn = sw;
        sw = tc; tc = tn; tn = sw;
        pc = pn;
    }
    if (part) {
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0)
            part[(int64_t)k * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

// ---------------------------------------------------------------------------------------
// Plain FP32 fused A, asynchronous staging, tile extent fixed at compile time. Same marching
// scheme as k_apply_A, but each time slice of x and phi arrives by cp.async copies (16-byte
// chunks for x) into a four-slice ring in shared memory, issued three slices ahead, so no
// registers hold staged data and a slice has two steps to land. Thread i < TX*TY owns tile
// site (i % TX, i / TX) and keeps that site's x(t), t_(t) and phi(t) in registers: its
// t_(t+1) reads the four x neighbours and its y(t) the four t_ neighbours from shared memory.
// The one-site-ring t_ sites are a second job of threads 0, 1, ... One barrier per step:
// step t writes t_(t+1) into the t_ buffer that y(t-1) read before the barrier, and reads
// t_(t), written before it; slice t+3 goes into the x buffer of slice t-1, last read before it.

constexpr int kA4Ring = 4;   // x and phi slices resident: t-1 .. t+2

template <int TX, int TY> struct A4Shape {
    static constexpr int HX2 = TX + 4, N2 = (TX + 4) * (TY + 4);   // two-site halo
    static constexpr int HX1 = TX + 2, N1 = (TX + 2) * (TY + 2);   // one-site halo
    static constexpr int NI = TX * TY;
    static constexpr int NCH = (2 * N2 + kAThreads - 1) / kAThreads;   // 16-byte chunks per thread and slice
    static constexpr int NPH = (N1 + kAThreads - 1) / kAThreads;       // phi sites per thread and slice
    static constexpr size_t smem = (size_t)kA4Ring * N2 * 32 + (size_t)2 * N1 * 32 + (size_t)kA4Ring * 3 * N1 * 4;
    static_assert(NI <= kAThreads && N1 - NI <= kAThreads, "one tile site and one ring site per thread");
};

template <int TX, int TY>
__global__ void __launch_bounds__(kAThreads, 2) k_apply_A4(Lat lat, Coef<float> cf, ATile tl,
                                                           const float* __restrict__ phi,
                                                           const Site<float>* __restrict__ x,
                                                           Site<float>* __restrict__ y, double* __restrict__ part,
                                                           const CgScalars* __restrict__ cgs) {
    if (cgs && !cgs[blockIdx.z].active) return;
    using S = A4Shape<TX, TY>;
    constexpr int HX2 = S::HX2, N2 = S::N2, HX1 = S::HX1, N1 = S::N1, NI = S::NI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint4* xsb = reinterpret_cast<uint4*>(smem_raw);                 // ring x [2 planes][N2]
    uint4* tsb = xsb + kA4Ring * 2 * N2;                             // 2 x [2 planes][N1]
    float* phb = reinterpret_cast<float*>(tsb + 2 * 2 * N1);         // ring x [3][N1]
    __shared__ double red[kAThreads / 32];

    const int L = lat.L, Nt = lat.Nt;
    const int64_t V = lat.V, LL = (int64_t)L * L;
    const int x0 = (blockIdx.x % tl.ntx) * TX, y0 = (blockIdx.x / tl.ntx) * TY;
    const int t0 = blockIdx.y * tl.C;
    const int t1 = min(t0 + tl.C, Nt);
    const int k = blockIdx.z;
    const Site<float>* xk = x + k * V;
    Site<float>* yk = y + k * V;
    auto gx = [&](int i) { int v = (x0 + i) % L; return v < 0 ? v + L : v; };
    auto gy = [&](int j) { int v = (y0 + j) % L; return v < 0 ? v + L : v; };
    auto wrap_t = [&](int t) { return t < 0 ? t + Nt : (t >= Nt ? t - Nt : t); };
    const int tid = threadIdx.x;

    // staging: chunk c = tid + j * threads is plane (c & 1) of two-site-halo site (c >> 1);
    // g_off in 16-byte units within a slice, -1 for none
    int g_off[S::NCH];
#pragma unroll
    for (int j = 0; j < S::NCH; ++j) {
        const int c = tid + j * kAThreads, i = c >> 1;
        g_off[j] = c < 2 * N2 ? 2 * (gy(i / HX2 - 2) * L + gx(i % HX2 - 2)) + (c & 1) : -1;
    }
    int p_off[S::NPH];
#pragma unroll
    for (int j = 0; j < S::NPH; ++j) {
        const int i = tid + j * kAThreads;
        p_off[j] = i < N1 ? gy(i / HX1 - 1) * L + gx(i % HX1 - 1) : -1;
    }
    // own tile site
    const bool own = tid < NI;
    const int ix = tid % TX, iy = tid / TX;
    const int o_c2 = (iy + 2) * HX2 + ix + 2, o_c1 = (iy + 1) * HX1 + ix + 1;
    const bool o_valid = own && x0 + ix < L && y0 + iy < L;
    const int o_off = gy(iy) * L + gx(ix);
    const float o_eta = ((gx(ix) + gy(iy)) & 1) ? -1.f : 1.f;
    // one-site-ring site of this thread: top row, the two side columns, bottom row
    int r1_c1 = -1, r1_c2 = 0;
    float r1_eta = 1.f;
    if (tid < N1 - NI) {
        int hx, hy;
        if (tid < HX1) { hy = 0; hx = tid; }
        else if (tid < HX1 + 2 * TY) { const int r = tid - HX1; hy = 1 + r / 2; hx = (r & 1) ? TX + 1 : 0; }
        else { hy = TY + 1; hx = tid - HX1 - 2 * TY; }
        r1_c1 = hy * HX1 + hx;
        r1_c2 = (hy + 1) * HX2 + hx + 1;
        r1_eta = ((gx(hx - 1) + gy(hy - 1)) & 1) ? -1.f : 1.f;
    }

    auto xbuf = [&](int b) { return xsb + b * (2 * N2); };
    auto tbuf = [&](int b) { return tsb + b * (2 * N1); };
    auto pbuf = [&](int b) { return phb + b * (3 * N1); };
    auto issue = [&](int b, int t) {
        const int64_t base = (int64_t)t * LL;
        const uint4* src = reinterpret_cast<const uint4*>(xk + base);
        uint4* dst = xbuf(b);
#pragma unroll
        for (int j = 0; j < S::NCH; ++j) {
            const int c = tid + j * kAThreads;
            if (g_off[j] >= 0) cp_async16(dst + (c & 1) * N2 + (c >> 1), src + g_off[j]);
        }
        float* pd = pbuf(b);
#pragma unroll
        for (int j = 0; j < S::NPH; ++j)
            if (p_off[j] >= 0) {
                const int i = tid + j * kAThreads;
                const float* ps = phi + base + p_off[j];
                cp_async4(pd + i, ps);
                cp_async4(pd + N1 + i, ps + V);
                cp_async4(pd + 2 * N1 + i, ps + 2 * V);
            }
    };
    // t_ at slice t on this thread's ring site from x(t) (buffer bc) and x(t-1) (buffer bp)
    auto ring_t = [&](int bc, int bp, int bt, int t) {
        if (r1_c1 < 0) return;
        const uint4* xc = xbuf(bc);
        const float* ph = pbuf(bc);
        const int c = r1_c2;
        const Site<float> o = site_op<float>(cf, sm_load<float>(xc, N2, c), sm_load<float>(xc, N2, c - 1),
                                             sm_load<float>(xc, N2, c + 1), sm_load<float>(xc, N2, c - HX2),
                                             sm_load<float>(xc, N2, c + HX2), sm_load<float>(xbuf(bp), N2, c),
                                             t == 0 ? -1.f : 1.f, ph[r1_c1], ph[N1 + r1_c1], ph[2 * N1 + r1_c1],
                                             r1_eta);
        sm_store<float>(tbuf(bt), N1, r1_c1, o);
    };
    // t_ at slice t on the own site from x(t) (buffer bc, also returned in xo) and x(t-1)
    auto own_t = [&](int bc, const Site<float>& xprev, int bt, int t, Site<float>& xo, float* ph3) {
        const uint4* xc = xbuf(bc);
        const float* ph = pbuf(bc);
        xo = sm_load<float>(xc, N2, o_c2);
        ph3[0] = ph[o_c1]; ph3[1] = ph[N1 + o_c1]; ph3[2] = ph[2 * N1 + o_c1];
        const Site<float> o = site_op<float>(cf, xo, sm_load<float>(xc, N2, o_c2 - 1), sm_load<float>(xc, N2, o_c2 + 1),
                                             sm_load<float>(xc, N2, o_c2 - HX2), sm_load<float>(xc, N2, o_c2 + HX2),
                                             xprev, t == 0 ? -1.f : 1.f, ph3[0], ph3[1], ph3[2], o_eta);
        sm_store<float>(tbuf(bt), N1, o_c1, o);
        return o;
    };

    // prologue: slices t0-1 .. t0+2 in buffers 0 .. 3 (slice t0+2 only if step t0+1 exists)
    issue(0, wrap_t(t0 - 1));
    cp_async_commit();
    issue(1, t0);
    cp_async_commit();
    issue(2, wrap_t(t0 + 1));   // y(t0) needs t_(t0+1) even when the chunk is one slice long
    cp_async_commit();
    if (t0 + 1 < t1) issue(3, wrap_t(t0 + 2));
    cp_async_commit();
    cp_async_wait<2>();
    __syncthreads();
    Site<float> xo, to;
    float pho[3] = {0.f, 0.f, 0.f};
    if (own) to = own_t(1, sm_load<float>(xbuf(0), N2, o_c2), 0, t0, xo, pho);
    ring_t(1, 0, 0, t0);

    float acc = 0.f;
    for (int t = t0; t < t1; ++t) {
        const int u = t - t0 + 1;              // ring buffer of slice t is u & 3
        cp_async_wait<1>();                    // slice t+1 has landed (slice t+2 may be in flight)
        __syncthreads();
        if (t + 2 < t1) issue((u + 3) & 3, wrap_t(t + 3));
        cp_async_commit();
        const int tp = wrap_t(t + 1);
        const int bn = (u + 1) & 3, bt = (t + 1 - t0) & 1;
        Site<float> xn, tn;
        float phn[3] = {0.f, 0.f, 0.f};
        if (own) tn = own_t(bn, xo, bt, tp, xn, phn);
        ring_t(bn, u & 3, bt, tp);
        // y(t) = D t_ on the own site: t_(t) neighbours from the buffer written before the barrier
        if (own) {
            const uint4* tc = tbuf(bt ^ 1);
            const Site<float> o = site_op<float>(cf, to, sm_load<float>(tc, N1, o_c1 - 1),
                                                 sm_load<float>(tc, N1, o_c1 + 1), sm_load<float>(tc, N1, o_c1 - HX1),
                                                 sm_load<float>(tc, N1, o_c1 + HX1), tn, t == Nt - 1 ? -1.f : 1.f,
                                                 pho[0], pho[1], pho[2], o_eta);
            if (o_valid) {
                store_site(yk + (int64_t)t * LL + o_off, o);
                if (part) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc += to.c[q].x * to.c[q].x + to.c[q].y * to.c[q].y;
                }
            }
            xo = xn;
            to = tn;
            pho[0] = phn[0]; pho[1] = phn[1]; pho[2] = phn[2];
        }
    }
    cp_async_wait<0>();
    if (part) {
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0)
            part[(int64_t)k * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

static int largest_divisor_le(int L, int cap) {
    for (int d = cap < L ? cap : L; d >= 1; --d)
        if (L % d == 0) return d;
    return 1;
}

static ATile choose_tile_sms(int num_sms, const Lat& lat, int nrhs, size_t site_bytes);
static ATile choose_tile(const hmc_ctx* ctx, const Lat& lat, int nrhs, size_t site_bytes) {
    return choose_tile_sms(ctx->num_sms, lat, nrhs, site_bytes);
}
static ATile choose_tile_sms(int num_sms, const Lat& lat, int nrhs, size_t site_bytes) {
    ATile t;
    t.TX = largest_divisor_le(lat.L, site_bytes > 32 ? 16 : 32);
    if (lat.L % 16 == 0 && site_bytes <= 32) t.TX = 16;
    int cap = (site_bytes > 32 ? 128 : 256) / t.TX;
    t.TY = largest_divisor_le(lat.L, cap < 1 ? 1 : cap);
    // each thread stages at most NPF two-site-ring sites (TY <= kAThreads / TX keeps the tile
    // within one output site per thread)
    const int n2max = (site_bytes > 32 ? 1 : 2) * kAThreads;
    while ((t.TX + 4) * (t.TY + 4) > n2max && t.TY > 1) t.TY = largest_divisor_le(lat.L, t.TY - 1);
    while ((t.TX + 4) * (t.TY + 4) > n2max && t.TX > 1) t.TX = largest_divisor_le(lat.L, t.TX - 1);
    t.ntx = (lat.L + t.TX - 1) / t.TX;
    t.nty = (lat.L + t.TY - 1) / t.TY;
    const int64_t tiles = (int64_t)t.ntx * t.nty * nrhs;
    const int64_t target = (int64_t)num_sms * 8;
    int C = (int)((lat.Nt * tiles + target - 1) / target);
    if (C < 4) C = 4;
    if (C > lat.Nt) C = lat.Nt;
    t.C = C;
    t.nchunk = (lat.Nt + C - 1) / C;
    return t;
}

template <typename R>
static size_t a_smem_bytes(const ATile& t) {
    const int N2 = (t.TX + 4) * (t.TY + 4), N1 = (t.TX + 2) * (t.TY + 2);
    return (size_t)2 * N2 * sizeof(Site<R>) + (size_t)2 * N1 * sizeof(Site<R>) + (size_t)9 * N1 * sizeof(R);
}

static ATile make_atile(const Lat& lat, int TX, int TY, int C) {
    ATile t;
    t.TX = TX;
    t.TY = TY;
    t.C = C < 1 ? 1 : (C > lat.Nt ? lat.Nt : C);
    t.ntx = (lat.L + TX - 1) / TX;
    t.nty = (lat.L + TY - 1) / TY;
    t.nchunk = (lat.Nt + t.C - 1) / t.C;
    return t;
}

// One launch of the fused A on tile tl: the plain FP32 operator takes the asynchronous-staging
// kernel where the tile fits it, everything else the register-prefetch kernel.
template <typename R>
static void go_apply_A(hmc_ctx* ctx, const Lat& lat, const ATile& tl, int nrhs, const R* phi, const Site<R>* x,
                       Site<R>* y, double* part, const CgScalars* cgs, const Site<R>* pold, Site<R>* pnew) {
    const dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
    const Coef<R> cf = make_coef<R>(ctx->p);
    if (pnew) {
        k_apply_A<R, true><<<grid, kAThreads, a_smem_bytes<R>(tl), ctx->stream>>>(lat, cf, tl, phi, x, y, part, cgs,
                                                                                  pold, pnew);
        return;
    }
    if constexpr (sizeof(R) == 4) {
        if (tl.TX == 16 && tl.TY == 16) {
            k_apply_A4<16, 16><<<grid, kAThreads, A4Shape<16, 16>::smem, ctx->stream>>>(lat, cf, tl, phi, x, y, part,
                                                                                        cgs);
            return;
        }
    }
    k_apply_A<R, false><<<grid, kAThreads, a_smem_bytes<R>(tl), ctx->stream>>>(lat, cf, tl, phi, x, y, part, cgs,
                                                                               nullptr, nullptr);
}

// Times every valid (TX, TY, C) on the call's own buffers (the launch is idempotent: y, pnew
// and the partial sums depend only on the inputs) and returns the fastest.
template <typename R>
static int autotune_A(hmc_ctx* ctx, const Lat& lat, const R* phi, const Site<R>* x, Site<R>* y, int nrhs,
                      double* part, const CgScalars* cgs, const Site<R>* pold, Site<R>* pnew, ATile* best) {
    const ATile base = *best;
    const int txmax = sizeof(R) == 8 ? 16 : 32, tmax = sizeof(R) == 8 ? 128 : kAThreads;
    std::vector<ATile> cand;
    for (int TX = 2; TX <= txmax && TX <= lat.L; ++TX) {
        if (lat.L % TX) continue;
        for (int TY = 2; TY <= lat.L && TX * TY <= tmax; ++TY) {
            if (lat.L % TY || (TX + 4) * (TY + 4) > (sizeof(R) == 8 ? 1 : 2) * kAThreads) continue;
            if (a_smem_bytes<R>(make_atile(lat, TX, TY, 1)) > 200 * 1024) continue;
            if (TX * TY < 32) continue;
            // time chunks around the one that gives ~8 blocks per SM: half, same, 2x, 4x
            const int64_t tiles = (int64_t)(lat.L / TX) * (lat.L / TY) * nrhs;
            const int64_t target = (int64_t)ctx->num_sms * 8;
            const int c0 = (int)((lat.Nt * tiles + target - 1) / target);
            int last = -1;
            for (int C : {c0 / 2, c0, 2 * c0, 4 * c0}) {
                C = C < 4 ? 4 : (C > lat.Nt ? lat.Nt : C);
                if (C == last) continue;
                last = C;
                cand.push_back(make_atile(lat, TX, TY, C));
            }
        }
    }
    if (cand.empty()) return HMC_OK;
    cudaEvent_t e0, e1;
    HMC_CUDA(ctx, cudaEventCreate(&e0));
    HMC_CUDA(ctx, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (const ATile& tl : cand) {
        const dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
        if (part && (int64_t)grid.x * grid.y * nrhs > ctx->part_cap) continue;
        auto go = [&]() { go_apply_A<R>(ctx, lat, tl, nrhs, phi, x, y, part, cgs, pold, pnew); };
        go();
        HMC_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 3; ++r) go();
        HMC_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        HMC_CUDA(ctx, cudaEventSynchronize(e1));
        HMC_LAUNCH(ctx, "k_apply_A (tuning)");
        float ms = 0.f;
        HMC_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; *best = tl; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)base;
    return HMC_OK;
}

template <typename R>
int launch_apply_A(hmc_ctx* ctx, const Lat& lat, const R* phi, const cplx<R>* x, cplx<R>* y,
                   int nrhs, double* part, int* nblk_out, const CgScalars* cgs,
                   const cplx<R>* pold, cplx<R>* pnew) {
    if (nrhs <= 0) return HMC_OK;
    if (pnew && (!cgs || !pold || pold == pnew)) return fail(ctx, HMC_ERR_ARG, "apply_A: bad direction-update buffers");
    if constexpr (sizeof(R) == 4) {
        if (!pnew && strip_supported(lat))
            return launch_apply_A_strip(ctx, lat, phi, x, y, nrhs, part, nblk_out, cgs);
    }
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        if constexpr (sizeof(R) == 4)
        {
            HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A4<16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)A4Shape<16, 16>::smem));
        }
        attr.mark(bit);
    }
    const int prec = sizeof(R) == 8 ? HMC_FP64 : HMC_FP32;
    ATile tl;
    bool found = false;
    for (const ATuned& a : ctx->atuned)
        if (a.L == lat.L && a.Nt == lat.Nt && a.nrhs == nrhs && a.prec == prec) {
            tl = make_atile(lat, a.TX, a.TY, a.C);
            found = true;
            break;
        }
    if (!found) {
        tl = choose_tile(ctx, lat, nrhs, sizeof(Site<R>));
        if (ctx->p.autotune) {
            int rc = autotune_A<R>(ctx, lat, phi, reinterpret_cast<const Site<R>*>(x), reinterpret_cast<Site<R>*>(y),
                                   nrhs, part, cgs, reinterpret_cast<const Site<R>*>(pold),
                                   reinterpret_cast<Site<R>*>(pnew), &tl);
            if (rc) return rc;
        }
        ctx->atuned.push_back(ATuned{lat.L, lat.Nt, nrhs, prec, tl.TX, tl.TY, tl.C});
    }
    dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
    if (part && (int64_t)grid.x * grid.y * nrhs > ctx->part_cap)
        return fail(ctx, HMC_ERR_ARG, "apply_A: reduction buffer too small");
    go_apply_A<R>(ctx, lat, tl, nrhs, phi, reinterpret_cast<const Site<R>*>(x), reinterpret_cast<Site<R>*>(y), part,
                  cgs, reinterpret_cast<const Site<R>*>(pold), reinterpret_cast<Site<R>*>(pnew));
    HMC_LAUNCH(ctx, "k_apply_A");
    if (nblk_out) *nblk_out = grid.x * grid.y;
    return HMC_OK;
}
template int launch_apply_A<float>(hmc_ctx*, const Lat&, const float*, const float2*, float2*, int, double*, int*,
                                   const CgScalars*, const float2*, float2*);
template int launch_apply_A<double>(hmc_ctx*, const Lat&, const double*, const double2*, double2*, int, double*, int*,
                                    const CgScalars*, const double2*, double2*);

// ---------------------------------------------------------------------------------------
// Allocation-free variant of apply_MdagM for callers that cannot allocate device memory at
// call time. The per-block partial sums of ||D^dagger x||^2 and their row sums live in
// file-scope device arrays of fixed size instead of context workspace.
constexpr int64_t kStaticPartials = 1 << 16;   // partial sums (doubles): 512 KiB per device
constexpr int kStaticRows = 64;                // reduced sums: nrhs <= 64
static __device__ __align__(256) double g_static_part[kStaticPartials];
static __device__ __align__(256) double g_static_rows[kStaticRows];

struct StaticScratch {
    double* part = nullptr;   // device addresses of the arrays above on one device
    double* rows = nullptr;
    int num_sms = 0;
};
static std::mutex g_static_mu;
static StaticScratch g_static[64];   // by device ordinal

// Device addresses of the static arrays on the current device, resolved once per device.
static int static_scratch(StaticScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "apply_MdagM_static: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticScratch& sc = g_static[dev];
    if (!sc.part) {
        void* a = nullptr;
        void* b = nullptr;
        if ((e = cudaGetSymbolAddress(&a, g_static_part)) != cudaSuccess)
            return cuda_check(nullptr, e, "apply_MdagM_static: cudaGetSymbolAddress");
        if ((e = cudaGetSymbolAddress(&b, g_static_rows)) != cudaSuccess)
            return cuda_check(nullptr, e, "apply_MdagM_static: cudaGetSymbolAddress");
        if ((e = cudaDeviceGetAttribute(&sc.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_check(nullptr, e, "apply_MdagM_static: device query");
        sc.rows = static_cast<double*>(b);
        sc.part = static_cast<double*>(a);
    }
    *out = &sc;
    return HMC_OK;
}

__global__ void __launch_bounds__(256) k_static_rows(const double* __restrict__ part, int nblk,
                                                     double* __restrict__ out) {
    __shared__ double red[8];
    const double* row = part + (int64_t)blockIdx.x * nblk;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += row[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

template <typename R>
static int apply_A_static(const hmc_params* p, const Lat& lat, const R* phi, const Site<R>* x, Site<R>* y,
                          int nrhs, double* norm2, cudaStream_t stream) {
    StaticScratch* sc = nullptr;
    int rc = static_scratch(&sc);
    if (rc) return rc;
    const ATile tl = choose_tile_sms(sc->num_sms, lat, nrhs, sizeof(Site<R>));
    const dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
    const int64_t nblk = (int64_t)grid.x * grid.y;
    if (norm2 && nblk * nrhs > kStaticPartials)
        return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: the norms need " + std::to_string(nblk * nrhs) +
                    " partial sums (" + std::to_string(nblk) + " tile blocks x " + std::to_string(nrhs) +
                    " right-hand sides), more than the " + std::to_string(kStaticPartials) + " slots of the static scratch");
    const size_t sm = a_smem_bytes<R>(tl);
    cudaError_t e = cudaFuncSetAttribute(k_apply_A<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "apply_MdagM_static: cudaFuncSetAttribute");
    k_apply_A<R, false><<<grid, kAThreads, sm, stream>>>(lat, make_coef<R>(*p), tl, phi, x, y,
                                                         norm2 ? sc->part : nullptr, nullptr, nullptr, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(nullptr, e, "apply_MdagM_static: k_apply_A");
    if (!norm2) return HMC_OK;
    k_static_rows<<<nrhs, 256, 0, stream>>>(sc->part, (int)nblk, sc->rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(nullptr, e, "apply_MdagM_static: k_static_rows");
    if ((e = cudaMemcpyAsync(norm2, sc->rows, nrhs * sizeof(double), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_check(nullptr, e, "apply_MdagM_static: copy of the norms");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_check(nullptr, e, "apply_MdagM_static: sync");
    return HMC_OK;
}

}  // namespace hmc

extern "C" int apply_MdagM_static(const hmc_params* p, int L, int Nt, int prec, const void* phi, const void* x,
                                  void* y, int nrhs, double* norm2, void* cuda_stream) {
    using namespace hmc;
    if (!p || !phi || !x || !y) return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: null argument");
    if ((((uintptr_t)phi) | ((uintptr_t)x) | ((uintptr_t)y)) & 15u)
        return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: pointer not 16-byte aligned");
    if (L < 2 || (L & 1) || L > 4096 || Nt < 2 || Nt > 65536)
        return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: need even L in [2, 4096] and Nt in [2, 65536]");
    if (nrhs < 1 || nrhs > 65535)
        return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: nrhs must be in [1, 65535]");
    if (norm2 && nrhs > kStaticRows)
        return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: nrhs must be at most 64 when norms are requested");
    if (prec != HMC_FP64 && prec != HMC_FP32) return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: unknown precision");
    Lat lat;
    lat.L = L;
    lat.Nt = Nt;
    lat.V = (int64_t)Nt * L * L;
    // y is written while x and phi are read: their byte ranges must be disjoint from y's
    const uintptr_t real_b = prec == HMC_FP64 ? 8 : 4;
    const uintptr_t vb = (uintptr_t)nrhs * (uintptr_t)lat.V * 8 * real_b, pb = 3 * (uintptr_t)lat.V * real_b;
    const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y, pa = (uintptr_t)phi;
    if (xa < ya + vb && ya < xa + vb) return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: x and y overlap");
    if (pa < ya + vb && ya < pa + pb) return fail(nullptr, HMC_ERR_ARG, "apply_MdagM_static: phi and y overlap");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HMC_FP64)
        return apply_A_static<double>(p, lat, (const double*)phi, (const Site<double>*)x, (Site<double>*)y, nrhs,
                                      norm2, st);
    if (prec == HMC_FP32)
        return apply_A_static<float>(p, lat, (const float*)phi, (const Site<float>*)x, (Site<float>*)y, nrhs,
                                     norm2, st);
    return HMC_ERR_ARG;
}

namespace hmc {

// ---------------------------------------------------------------------------------------
// Boson pieces: -dS_B/dphi and the S_B density of the forward-difference lattice action
// S_B = dtau sum [(1/c^2)|phi(t+1) - phi(t)|^2 / dtau^2 + (1/2) sum_d |phi(r+d) - phi(r)|^2 + (r/2)|phi|^2 + (u/4)|phi|^4].
struct BosonCoef {
    double dtau, kt, r, u;   // kt = 1 / (c^2 dtau^2)
};

__device__ __forceinline__ void boson_site(const Lat& lat, const BosonCoef& bc,
                                           const double* __restrict__ phi, int64_t s, int xx,
                                           int yy, int t, double F[3], double& dens) {
    const int L = lat.L;
    const int64_t V = lat.V, LL = (int64_t)L * L;
    const int64_t row = s - xx, slice = (int64_t)t * LL, inplane = s - slice;
    const int64_t sxp = row + wrap_inc(xx, L), sxm = row + wrap_dec(xx, L);
    const int64_t syp = slice + (int64_t)wrap_inc(yy, L) * L + xx;
    const int64_t sym = slice + (int64_t)wrap_dec(yy, L) * L + xx;
    const int64_t stp = (int64_t)tnext(t, lat.Nt) * LL + inplane;
    const int64_t stm = (int64_t)tprev(t, lat.Nt) * LL + inplane;
    double p[3], q2 = 0.0, kin = 0.0, grad = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) { p[a] = __ldg(phi + a * V + s); q2 += p[a] * p[a]; }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double* pa = phi + a * V;
        const double ptp = __ldg(pa + stp), ptm = __ldg(pa + stm);
        const double pxp = __ldg(pa + sxp), pxm = __ldg(pa + sxm);
        const double pyp = __ldg(pa + syp), pym = __ldg(pa + sym);
        const double dtp = ptp - p[a], dxp = pxp - p[a], dyp = pyp - p[a];
        kin += dtp * dtp;
        grad += dxp * dxp + dyp * dyp;
        const double lap_t = 2.0 * p[a] - ptp - ptm;
        const double lap_xy = 4.0 * p[a] - pxp - pxm - pyp - pym;
        F[a] = -bc.dtau * (2.0 * bc.kt * lap_t + lap_xy + bc.r * p[a] + bc.u * q2 * p[a]);
    }
    dens = bc.dtau * (bc.kt * kin + 0.5 * grad + 0.5 * bc.r * q2 + 0.25 * bc.u * q2 * q2);
}

// Force: F = -dS_B/dphi (optional) + sum_k 2 dtau g eta Re[X^dag (sigma^x (x) sigma^a) Y],
// Y = D^dagger X computed on the fly, or read from Yin when a solve's last true-residual
// evaluation left it (the same stencil on the same X, so the same bits, without the FP64 work).
// Partials: [0, nblk) = sum_k 2 Re<pf, X> - |Y|^2, [nblk, 2 nblk) = S_B density.
__global__ void __launch_bounds__(256) k_force(Lat lat, Coef<double> cf, BosonCoef bc,
                                               const double* __restrict__ phi,
                                               const Site<double>* __restrict__ X,
                                               const Site<double>* __restrict__ pf, int nrhs,
                                               double* __restrict__ F, int include_boson,
                                               double* __restrict__ part, const Site<double>* __restrict__ Yin) {
    __shared__ double red[8];
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double spf = 0.0, sb = 0.0;
    if (s < lat.V) {
        const int64_t V = lat.V;
        const int L = lat.L;
        const int xx = (int)(s % L);
        const int64_t rest = s / L;
        const int yy = (int)(rest % L);
        const int t = (int)(rest / L);
        const int64_t row = s - xx, slice = (int64_t)t * L * L;
        const int64_t sxm = row + wrap_dec(xx, L), sxp = row + wrap_inc(xx, L);
        const int64_t sym = slice + (int64_t)wrap_dec(yy, L) * L + xx;
        const int64_t syp = slice + (int64_t)wrap_inc(yy, L) * L + xx;
        const int64_t stm = (int64_t)tprev(t, lat.Nt) * L * L + (s - slice);
        const double tsign = t == 0 ? -1.0 : 1.0;
        const double eta = ((xx + yy) & 1) ? -1.0 : 1.0;
        const double p1 = __ldg(phi + s), p2 = __ldg(phi + V + s), p3 = __ldg(phi + 2 * V + s);
        double acc[3] = {0.0, 0.0, 0.0};
        auto ld = [&](const Site<double>* base, int64_t i) {
            Site<double> z{};
            return HMC_IN(i >= 0 && i < V, kBndForce) ? load_site(base + i) : z;
        };
        for (int k = 0; k < nrhs; ++k) {
            const Site<double>* Xk = X + k * V;
            const Site<double> xc = ld(Xk, s);
            const Site<double> Y = Yin ? ld(Yin + k * V, s)
                                       : site_op<double>(cf, xc, ld(Xk, sxm), ld(Xk, sxp), ld(Xk, sym), ld(Xk, syp),
                                                         ld(Xk, stm), tsign, p1, p2, p3, eta);
            const Site<double> pk = load_site(pf + k * V + s);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double2 x0 = xc.c[a * 2], x1 = xc.c[a * 2 + 1];
                const double2 y0 = Y.c[(1 - a) * 2], y1 = Y.c[(1 - a) * 2 + 1];
                const double2 z01 = cmulconj(x0, y1), z10 = cmulconj(x1, y0);
                const double2 z00 = cmulconj(x0, y0), z11 = cmulconj(x1, y1);
                acc[0] += z01.x + z10.x;          // sigma^1
                acc[1] += z01.y - z10.y;          // sigma^2: Re(-i z01 + i z10)
                acc[2] += z00.x - z11.x;          // sigma^3
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                spf += 2.0 * (pk.c[q].x * xc.c[q].x + pk.c[q].y * xc.c[q].y)
                       - (Y.c[q].x * Y.c[q].x + Y.c[q].y * Y.c[q].y);
            }
        }
        const double f = 2.0 * cf.cpl * eta;
        double Fb[3] = {0.0, 0.0, 0.0};
        if (include_boson) boson_site(lat, bc, phi, s, xx, yy, t, Fb, sb);
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a * V + s] = f * acc[a] + Fb[a];
    }
    const double a = block_sum(spf, red);
    const double b = block_sum(sb, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[gridDim.x + blockIdx.x] = b;
    }
}

static BosonCoef boson_coef(const hmc_params& p, double r) {
    BosonCoef b;
    b.dtau = p.dtau;
    b.kt = 1.0 / (p.c * p.c * p.dtau * p.dtau);
    b.r = r;
    b.u = p.u;
    return b;
}

int launch_force(hmc_ctx* ctx, const Lat& lat, double r, const double* phi, const double2* X,
                 const double2* pf, int nrhs, double* F, int include_boson, double* part,
                 int* nblk_out, const double2* Y) {
    const int nblk = (int)((lat.V + 255) / 256);
    if (2 * (int64_t)nblk > ctx->part_cap) return fail(ctx, HMC_ERR_ARG, "force: reduction buffer too small");
    k_force<<<nblk, 256, 0, ctx->stream>>>(lat, make_coef<double>(ctx->p), boson_coef(ctx->p, r), phi,
                                           reinterpret_cast<const Site<double>*>(X),
                                           reinterpret_cast<const Site<double>*>(pf), nrhs, F,
                                           include_boson, part, reinterpret_cast<const Site<double>*>(Y));
    HMC_LAUNCH(ctx, "k_force");
    *nblk_out = nblk;
    return HMC_OK;
}

__global__ void __launch_bounds__(256) k_boson(Lat lat, BosonCoef bc, const double* __restrict__ phi,
                                               double* __restrict__ F, double* __restrict__ part) {
    __shared__ double red[8];
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double sb = 0.0;
    if (s < lat.V) {
        const int L = lat.L;
        const int xx = (int)(s % L);
        const int64_t rest = s / L;
        double Fb[3];
        boson_site(lat, bc, phi, s, xx, (int)(rest % L), (int)(rest / L), Fb, sb);
        if (F) {
#pragma unroll
            for (int a = 0; a < 3; ++a) F[a * lat.V + s] = Fb[a];
        }
    }
    const double b = block_sum(sb, red);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

int launch_boson(hmc_ctx* ctx, const Lat& lat, double r, const double* phi, double* F,
                 double* part, int* nblk_out) {
    const int nblk = (int)((lat.V + 255) / 256);
    if (nblk > ctx->part_cap) return fail(ctx, HMC_ERR_ARG, "boson: reduction buffer too small");
    k_boson<<<nblk, 256, 0, ctx->stream>>>(lat, boson_coef(ctx->p, r), phi, F, part);
    HMC_LAUNCH(ctx, "k_boson");
    *nblk_out = nblk;
    return HMC_OK;
}

}  // namespace hmc

namespace hmc {
unsigned int bounds_take_stencil() { return bounds_take_tu(); }
}  // namespace hmc
