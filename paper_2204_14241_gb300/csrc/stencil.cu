// Fermion-matrix stencils (Eq. D_formula), the fused normal operator A = D D^dagger
// (Eq. linsys), and the fused force kernel (Eq. hamiltonseq with S = S_B + S_PF).
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
                                                 Site<R>* __restrict__ y) {
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
    Site<R> o = site_op<R>(cf, load_site(xk + s), load_site(xk + row + wrap_dec(xx, L)),
                           load_site(xk + row + wrap_inc(xx, L)),
                           load_site(xk + slice + (int64_t)wrap_dec(yy, L) * L + xx),
                           load_site(xk + slice + (int64_t)wrap_inc(yy, L) * L + xx),
                           load_site(xk + (int64_t)tn * L * L + (s - slice)), tsign,
                           __ldg(phi + s), __ldg(phi + V + s), __ldg(phi + 2 * V + s), eta);
    store_site(y + blockIdx.y * V + s, o);
}

template <typename R>
int launch_apply_D(hmc_ctx* ctx, const Lat& lat, const R* phi, const cplx<R>* x, cplx<R>* y,
                   int dagger, int nrhs) {
    if (nrhs <= 0) return HMC_OK;
    dim3 grid((unsigned)((lat.V + 255) / 256), nrhs);
    Coef<R> cf = make_coef<R>(ctx->p);
    auto xs = reinterpret_cast<const Site<R>*>(x);
    auto ys = reinterpret_cast<Site<R>*>(y);
    if (dagger) k_apply_D<R, true><<<grid, 256, 0, ctx->stream>>>(lat, cf, phi, xs, ys);
    else        k_apply_D<R, false><<<grid, 256, 0, ctx->stream>>>(lat, cf, phi, xs, ys);
    HMC_LAUNCH(ctx, "k_apply_D");
    return HMC_OK;
}
template int launch_apply_D<float>(hmc_ctx*, const Lat&, const float*, const float2*, float2*, int, int);
template int launch_apply_D<double>(hmc_ctx*, const Lat&, const double*, const double2*, double2*, int, int);

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

// With pnew != nullptr the kernel also performs the CG direction update: the operand is
// p = x + beta_k * pold (x holding z), formed as it is loaded, and the block writes p for the
// sites it owns (tile interior, slices [t0, t1)) to pnew; y = A p. pold and pnew must differ.
//
// Thread roles: thread i < TX*TY owns tile site (i % TX, i / TX) and keeps that site's x(t),
// t_(t) and t_(t+1) in registers, so its t_ and y need only the four spatial neighbours from
// shared memory. The remaining sites of the two-site ring (x staging) and of the one-site ring
// (t_ outputs, phi) are a second slot handled by threads 0, 1, ...
template <typename R>
__global__ void __launch_bounds__(kAThreads, sizeof(R) == 4 ? 2 : 1) k_apply_A(Lat lat, Coef<R> cf, ATile tl,
                                                          const R* __restrict__ phi,
                                                          const Site<R>* __restrict__ x,
                                                          Site<R>* __restrict__ y, double* __restrict__ part,
                                                          const CgScalars* __restrict__ cgs,
                                                          const Site<R>* __restrict__ pold,
                                                          Site<R>* __restrict__ pnew) {
    if (cgs && !cgs[blockIdx.z].active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = tl.TX, TY = tl.TY;
    const int HX2 = TX + 4, HY2 = TY + 4, N2 = HX2 * HY2;
    const int HX1 = TX + 2, HY1 = TY + 2, N1 = HX1 * HY1;
    const int NI = TX * TY;
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
    const R beta = pnew ? (R)cgs[k].beta : R(0);
    const Site<R>* pok = pnew ? pold + k * V : nullptr;
    Site<R>* pnk = pnew ? pnew + k * V : nullptr;
    auto gx = [&](int i) { int v = (x0 + i) % L; return v < 0 ? v + L : v; };
    auto gy = [&](int j) { int v = (y0 + j) % L; return v < 0 ? v + L : v; };

    // ---- per-thread geometry, fixed for the whole march ------------------------------------
    const int tid = threadIdx.x;
    // slot 0: own tile site
    const bool own = tid < NI;
    int o_ix = 0, o_iy = 0, o_off = -1, o_c2 = 0, o_c1 = 0;
    R o_eta = R(1);
    bool o_valid = false;   // inside the lattice (ragged tiles)
    if (own) {
        o_ix = tid % TX;
        o_iy = tid / TX;
        const int X = gx(o_ix), Y = gy(o_iy);
        o_valid = x0 + o_ix < L && y0 + o_iy < L;
        o_off = Y * L + X;
        o_c2 = (o_iy + 2) * HX2 + o_ix + 2;
        o_c1 = (o_iy + 1) * HX1 + o_ix + 1;
        o_eta = ((X + Y) & 1) ? R(-1) : R(1);
    }
    // slot 1 of the two-site ring (x staging): ring sites in row-major order
    int r2_off = -1, r2_c = 0;
    bool r2_outer = false;
    {
        const int q = tid;
        if (q < N2 - NI) {
            int hx, hy;
            if (q < 2 * HX2) { hy = q / HX2; hx = q % HX2; }
            else if (q < 2 * HX2 + 4 * TY) { const int r = q - 2 * HX2; hy = 2 + r / 4; const int c = r % 4; hx = c < 2 ? c : TX + c; }
            else { const int r = q - 2 * HX2 - 4 * TY; hy = TY + 2 + r / HX2; hx = r % HX2; }
            r2_off = gy(hy - 2) * L + gx(hx - 2);
            r2_c = hy * HX2 + hx;
            r2_outer = hx == 0 || hy == 0 || hx == HX2 - 1 || hy == HY2 - 1;
        }
    }
    // slot 1 of the one-site ring (t_ outputs and phi)
    int r1_off = -1, r1_c1 = 0, r1_c2 = 0;
    R r1_eta = R(1);
    {
        const int q = tid;
        if (q < N1 - NI) {
            int hx, hy;
            if (q < HX1) { hy = 0; hx = q; }
            else if (q < HX1 + 2 * TY) { const int r = q - HX1; hy = 1 + r / 2; hx = (r % 2) ? TX + 1 : 0; }
            else { const int r = q - HX1 - 2 * TY; hy = TY + 1; hx = r; }
            const int X = gx(hx - 1), Y = gy(hy - 1);
            r1_off = Y * L + X;
            r1_c1 = hy * HX1 + hx;
            r1_c2 = (hy + 1) * HX2 + hx + 1;
            r1_eta = ((X + Y) & 1) ? R(-1) : R(1);
        }
    }

    // ---- register prefetch of one slice ------------------------------------------------------
    Site<R> rz0, rp0, rz1, rp1;
    R ph0[3], ph1[3];
    auto fetch = [&](int t) {
        const int64_t base = (int64_t)t * LL;
        if (own) {
            rz0 = load_site(xk + base + o_off);
            if (pnew) rp0 = load_site(pok + base + o_off);
            const R* pp = phi + base + o_off;
            ph0[0] = __ldg(pp); ph0[1] = __ldg(pp + V); ph0[2] = __ldg(pp + 2 * V);
        }
        if (r2_off >= 0) {
            rz1 = load_site(xk + base + r2_off);
            if (pnew) rp1 = load_site(pok + base + r2_off);
        }
        if (r1_off >= 0) {
            const R* pp = phi + base + r1_off;
            ph1[0] = __ldg(pp); ph1[1] = __ldg(pp + V); ph1[2] = __ldg(pp + 2 * V);
        }
    };
    auto combine = [&](Site<R> v, const Site<R>& po) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v.c[q].x += beta * po.c[q].x;
            v.c[q].y += beta * po.c[q].y;
        }
        return v;
    };
    // Store the prefetched slice t into dst / ph; returns the own site's value. ring1only
    // skips the outermost ring (slice t0 - 1 is needed on the one-site ring only).
    auto commit = [&](uint4* dst, R* ph, int t, bool own_write, bool ring1only) -> Site<R> {
        const int64_t base = (int64_t)t * LL;
        Site<R> v0 = rz0;
        if (own) {
            if (pnew) {
                v0 = combine(rz0, rp0);
                if (own_write && o_valid) store_site(pnk + base + o_off, v0);
            }
            sm_store<R>(dst, N2, o_c2, v0);
            if (ph) { ph[o_c1] = ph0[0]; ph[N1 + o_c1] = ph0[1]; ph[2 * N1 + o_c1] = ph0[2]; }
        }
        if (r2_off >= 0 && !(ring1only && r2_outer)) {
            const Site<R> v1 = pnew ? combine(rz1, rp1) : rz1;
            sm_store<R>(dst, N2, r2_c, v1);
        }
        if (r1_off >= 0 && ph) { ph[r1_c1] = ph1[0]; ph[N1 + r1_c1] = ph1[1]; ph[2 * N1 + r1_c1] = ph1[2]; }
        return v0;
    };

    // ---- prologue: x(t0), x(t0 - 1), t_(t0) ------------------------------------------------
    fetch(t0);
    Site<R> xo_cur = commit(xa, phb, t0, true, false);         // x(t0) at the own site
    R pho_cur[3] = {ph0[0], ph0[1], ph0[2]};                  // phi(t0) at the own site
    fetch(tprev(t0, Nt));
    const Site<R> xo_prev = commit(xb, nullptr, tprev(t0, Nt), false, true);
    __syncthreads();
    Site<R> to_cur;                                             // t_(t0) at the own site
    {
        const R tsign = (t0 == 0) ? R(-1) : R(1);
        if (own) {
            to_cur = site_op<R>(cf, xo_cur, sm_load<R>(xa, N2, o_c2 - 1), sm_load<R>(xa, N2, o_c2 + 1),
                                sm_load<R>(xa, N2, o_c2 - HX2), sm_load<R>(xa, N2, o_c2 + HX2), xo_prev, tsign,
                                pho_cur[0], pho_cur[1], pho_cur[2], o_eta);
            sm_store<R>(ta, N1, o_c1, to_cur);
        }
        if (r1_off >= 0) {
            const int c = r1_c2;
            const Site<R> o = site_op<R>(cf, sm_load<R>(xa, N2, c), sm_load<R>(xa, N2, c - 1),
                                         sm_load<R>(xa, N2, c + 1), sm_load<R>(xa, N2, c - HX2),
                                         sm_load<R>(xa, N2, c + HX2), sm_load<R>(xb, N2, c), tsign,
                                         phb[r1_c1], phb[N1 + r1_c1], phb[2 * N1 + r1_c1], r1_eta);
            sm_store<R>(ta, N1, r1_c1, o);
        }
    }
    fetch(tnext(t0, Nt));
    __syncthreads();

    // ---- march -------------------------------------------------------------------------------
    uint4 *xc = xa, *xn = xb, *tc = ta, *tn = tb;
    int pc = 0;   // phi(t) is in buffer pc of the three at phb
    R acc = 0;    // per-thread partial of ||D^dagger x||^2, in the operator's precision
    for (int t = t0; t < t1; ++t) {
        const int tp = tnext(t, Nt);
        const int pn = pc == 2 ? 0 : pc + 1;
        R* phn = phb + pn * 3 * N1;
        const Site<R> xo_next = commit(xn, phn, tp, t + 1 < t1, false);
        const R pho_next[3] = {ph0[0], ph0[1], ph0[2]};
        if (t + 1 < t1) fetch(tnext(tp, Nt));
        __syncthreads();
        // t_(t+1) = D^dagger x at slice t+1 on the one-site ring
        const R tsg = (tp == 0) ? R(-1) : R(1);   // b(t)
        Site<R> to_next;
        if (own) {
            to_next = site_op<R>(cf, xo_next, sm_load<R>(xn, N2, o_c2 - 1), sm_load<R>(xn, N2, o_c2 + 1),
                                 sm_load<R>(xn, N2, o_c2 - HX2), sm_load<R>(xn, N2, o_c2 + HX2), xo_cur, tsg,
                                 pho_next[0], pho_next[1], pho_next[2], o_eta);
            sm_store<R>(tn, N1, o_c1, to_next);
        }
        if (r1_off >= 0) {
            const int c = r1_c2;
            const Site<R> o = site_op<R>(cf, sm_load<R>(xn, N2, c), sm_load<R>(xn, N2, c - 1),
                                         sm_load<R>(xn, N2, c + 1), sm_load<R>(xn, N2, c - HX2),
                                         sm_load<R>(xn, N2, c + HX2), sm_load<R>(xc, N2, c), tsg,
                                         phn[r1_c1], phn[N1 + r1_c1], phn[2 * N1 + r1_c1], r1_eta);
            sm_store<R>(tn, N1, r1_c1, o);
        }
        __syncthreads();
        // y(t) = D t_ on the tile
        if (own) {
            const R tsign = (t == Nt - 1) ? R(-1) : R(1);   // b(t)
            const int c = o_c1;
            const Site<R> o = site_op<R>(cf, to_cur, sm_load<R>(tc, N1, c - 1), sm_load<R>(tc, N1, c + 1),
                                         sm_load<R>(tc, N1, c - HX1), sm_load<R>(tc, N1, c + HX1), to_next, tsign,
                                         pho_cur[0], pho_cur[1], pho_cur[2], o_eta);
            if (o_valid) {
                store_site(yk + (int64_t)t * LL + o_off, o);
                if (part) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc += to_cur.c[q].x * to_cur.c[q].x + to_cur.c[q].y * to_cur.c[q].y;
                }
            }
            xo_cur = xo_next;
            to_cur = to_next;
            pho_cur[0] = pho_next[0]; pho_cur[1] = pho_next[1]; pho_cur[2] = pho_next[2];
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

static int largest_divisor_le(int L, int cap) {
    for (int d = cap < L ? cap : L; d >= 1; --d)
        if (L % d == 0) return d;
    return 1;
}

static ATile choose_tile(const hmc_ctx* ctx, const Lat& lat, int nrhs, size_t site_bytes) {
    ATile t;
    t.TX = largest_divisor_le(lat.L, site_bytes > 32 ? 16 : 32);
    if (lat.L % 16 == 0 && site_bytes <= 32) t.TX = 16;
    int cap = (site_bytes > 32 ? 128 : 256) / t.TX;
    t.TY = largest_divisor_le(lat.L, cap < 1 ? 1 : cap);
    // one tile site per thread (TY <= kAThreads / TX) and at most one ring site per thread
    auto ring2 = [](const ATile& a) { return 4 * (a.TX + 4) + 4 * a.TY; };
    while (ring2(t) > kAThreads && t.TY > 1) t.TY = largest_divisor_le(lat.L, t.TY - 1);
    while (ring2(t) > kAThreads && t.TX > 1) t.TX = largest_divisor_le(lat.L, t.TX - 1);
    t.ntx = (lat.L + t.TX - 1) / t.TX;
    t.nty = (lat.L + t.TY - 1) / t.TY;
    const int64_t tiles = (int64_t)t.ntx * t.nty * nrhs;
    const int64_t target = (int64_t)ctx->num_sms * 8;
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
            if (lat.L % TY || 4 * (TX + 4) + 4 * TY > kAThreads) continue;
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
    const Coef<R> cf = make_coef<R>(ctx->p);
    for (const ATile& tl : cand) {
        const dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
        if (part && (int64_t)grid.x * grid.y * nrhs > ctx->part_cap) continue;
        const size_t sm = a_smem_bytes<R>(tl);
        k_apply_A<R><<<grid, kAThreads, sm, ctx->stream>>>(lat, cf, tl, phi, x, y, part, cgs, pold, pnew);
        HMC_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 3; ++r)
            k_apply_A<R><<<grid, kAThreads, sm, ctx->stream>>>(lat, cf, tl, phi, x, y, part, cgs, pold, pnew);
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
    static bool attr_set[2] = {false, false};
    if (!attr_set[sizeof(R) == 8]) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr_set[sizeof(R) == 8] = true;
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
    const size_t sm = a_smem_bytes<R>(tl);
    dim3 grid(tl.ntx * tl.nty, tl.nchunk, nrhs);
    if (part && (int64_t)grid.x * grid.y * nrhs > ctx->part_cap)
        return fail(ctx, HMC_ERR_ARG, "apply_A: reduction buffer too small");
    k_apply_A<R><<<grid, kAThreads, sm, ctx->stream>>>(lat, make_coef<R>(ctx->p), tl, phi,
                                                 reinterpret_cast<const Site<R>*>(x),
                                                 reinterpret_cast<Site<R>*>(y), part, cgs,
                                                 reinterpret_cast<const Site<R>*>(pold),
                                                 reinterpret_cast<Site<R>*>(pnew));
    HMC_LAUNCH(ctx, "k_apply_A");
    if (nblk_out) *nblk_out = grid.x * grid.y;
    return HMC_OK;
}
template int launch_apply_A<float>(hmc_ctx*, const Lat&, const float*, const float2*, float2*, int, double*, int*,
                                   const CgScalars*, const float2*, float2*);
template int launch_apply_A<double>(hmc_ctx*, const Lat&, const double*, const double2*, double2*, int, double*, int*,
                                    const CgScalars*, const double2*, double2*);

// ---------------------------------------------------------------------------------------
// Boson pieces: -dS_B/dphi and the S_B density (forward differences, see oracle reading).
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
// Y = D^dagger X computed on the fly. Partials: [0, nblk) = sum_k 2 Re<pf, X> - |Y|^2,
// [nblk, 2 nblk) = S_B density.
__global__ void __launch_bounds__(256) k_force(Lat lat, Coef<double> cf, BosonCoef bc,
                                               const double* __restrict__ phi,
                                               const Site<double>* __restrict__ X,
                                               const Site<double>* __restrict__ pf, int nrhs,
                                               double* __restrict__ F, int include_boson,
                                               double* __restrict__ part) {
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
        for (int k = 0; k < nrhs; ++k) {
            const Site<double>* Xk = X + k * V;
            const Site<double> xc = load_site(Xk + s);
            const Site<double> Y = site_op<double>(cf, xc, load_site(Xk + sxm), load_site(Xk + sxp),
                                                   load_site(Xk + sym), load_site(Xk + syp),
                                                   load_site(Xk + stm), tsign, p1, p2, p3, eta);
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
                 int* nblk_out) {
    const int nblk = (int)((lat.V + 255) / 256);
    if (2 * (int64_t)nblk > ctx->part_cap) return fail(ctx, HMC_ERR_ARG, "force: reduction buffer too small");
    k_force<<<nblk, 256, 0, ctx->stream>>>(lat, make_coef<double>(ctx->p), boson_coef(ctx->p, r), phi,
                                           reinterpret_cast<const Site<double>*>(X),
                                           reinterpret_cast<const Site<double>*>(pf), nrhs, F,
                                           include_boson, part);
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
