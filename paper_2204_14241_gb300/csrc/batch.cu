// Batched solves of many uneven lattices in one persistent launch.
//
// Every (chain, right-hand side) pair of a context solves A X = varphi (Eq. linsys) with the
// mixed-precision CG of cg.cu (complex64 iterations, FP64 solution and true residual, reliable
// updates when the iterated residual has dropped by 1e3, stop on the FP64 true residual), all
// pairs inside ONE cooperative launch: a grid-wide barrier separates the phases of an iteration,
// and pairs that have converged stop contributing. The vectors of all pairs are concatenated,
// chain c's K right-hand sides at item offset off_c ([c][k][site], 4 complex per item).
//
// Work is split into tiles of kTile sites of one pair, dealt round-robin to the blocks; every
// reduction is per tile (block-level, fixed order) and then per pair by one block (fixed order),
// so the results are reproducible bit for bit. Phases of one iteration:
//   I   p = r + beta p_old formed at each site and its neighbours on the fly, t_ = D^dagger p,
//       partial <p, A p> = ||t_||^2;                                               | barrier
//   III alpha = <r, r> / <p, A p> of the tile's pair (formed by every block that needs it, in
//       the same order), q = D t_ (never stored), x += alpha p, r -= alpha q, partial ||r||^2;
//                                                                                   | barrier
//   IV  beta, convergence and the reliable-update request per pair;                 | barrier
// and, when some pair asks for it, a reliable update: x64 += x32, x32 = 0 | t64 = D^dagger x64 |
// r64 = b - D t64, r32 = r64, partial ||r64||^2 | per pair: converged pairs stop.
// When the launch ends, t64 holds D^dagger x64 of every pair's returned solution (from the pair's last
// true residual, or the start), which the force reuses.
// The grid barrier spins on a generation word with a time limit (globaltimer); a block that gives
// up sets the error word, and since it never arrives at the next barrier every other block gives
// up there too: the launch ends and the host reports HMC_ERR_TIMEOUT.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace hmc {

constexpr int kBThreads = 256;
constexpr int kTile = 1024;   // sites per tile

struct BScal {
    double rr, pAp, alpha, beta, r2, r2_max, b2, r2true;
    int active, iters, need_ru, nonfinite;
};

struct BTile {
    int pair;       // chain * K + k
    int chain;
    int s0, s1;     // site range within the pair's vector
};

struct BatchArgs {
    int nchains, K, ntiles, npairs;
    const BChainDev* ch;
    const BTile* tiles;
    const int* pair_t0;     // first tile of each pair (npairs + 1 entries)
    Coef<float> cf32;
    Coef<double> cf64;
    const Site<double>* b;
    Site<double>* x64;
    Site<double>* r64;
    Site<double>* t64;
    Site<float>* x32;
    Site<float>* r32;
    Site<float>* pA;
    Site<float>* pB;
    Site<float>* t32;
    BScal* sc;
    double* part;           // [ntiles][2]
    unsigned* bar;          // [0] arrivals, [1] generation
    int* flags;             // [0] error word; [1] reliable update requested
    int* nactive;           // pairs still iterating
    int* iters_out;         // [0] iterations of the slowest pair, [1] reliable updates
    double tol2, delta2;
    int maxit, use_x0, test_timeout;
    long long timeout_ns;
};

// Vectors and scalars written inside the launch by other blocks are read through L2 (ld.cg): the
// per-SM L1 is not coherent across blocks. Inputs that no block writes use the read-only path.
template <typename R> __device__ __forceinline__ Site<R> ldcg_site(const Site<R>* p);
template <> __device__ __forceinline__ Site<float> ldcg_site<float>(const Site<float>* p) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldcg(q), b = __ldcg(q + 1);
    Site<float> s;
    s.c[0] = make_float2(a.x, a.y); s.c[1] = make_float2(a.z, a.w);
    s.c[2] = make_float2(b.x, b.y); s.c[3] = make_float2(b.z, b.w);
    return s;
}
template <> __device__ __forceinline__ Site<double> ldcg_site<double>(const Site<double>* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    Site<double> s;
    s.c[0] = __ldcg(q); s.c[1] = __ldcg(q + 1); s.c[2] = __ldcg(q + 2); s.c[3] = __ldcg(q + 3);
    return s;
}
__device__ __forceinline__ int ldcg_int(const int* p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_dbl(const double* p) { return __ldcg(p); }

__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a time limit. Returns false (and sets flags[0]) when it gives up.
__device__ bool grid_sync(const BatchArgs& a, bool never) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = a.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned target = gridDim.x + (never ? 1u : 0u);   // never: a count nothing reaches
        const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
        if (arrived == target) {
            atomicExch(a.bar, 0u);
            __threadfence();
            atomicAdd(const_cast<unsigned*>(gen), 1u);
        } else {
            const long long t0 = gtimer();
            while (*gen == g) {
                if (gtimer() - t0 > a.timeout_ns) {
                    ok = 0;
                    atomicOr(a.flags, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ void site_coords(const BChainDev& c, int s, int& xx, int& yy, int& t) {
    t = (int)(((float)s + 0.5f) * c.invLL);
    const int rem = s - t * c.LL;
    yy = (int)(((float)rem + 0.5f) * c.invL);
    xx = rem - yy * c.L;
}

// Neighbour site indices of s: x-1, x+1, y-1, y+1 and the time neighbour (t+1 for D, t-1 for D^dagger)
struct Nbr {
    int c, xm, xp, ym, yp, tn;
    bool wrap_sign;   // the time hop crosses the antiperiodic boundary
};
__device__ __forceinline__ Nbr neighbours(const BChainDev& c, int s, bool dag) {
    int xx, yy, t;
    site_coords(c, s, xx, yy, t);
    Nbr n;
    const int row = s - xx, slice = t * c.LL;
    n.c = s;
    n.xm = row + (xx == 0 ? c.L - 1 : xx - 1);
    n.xp = row + (xx == c.L - 1 ? 0 : xx + 1);
    n.ym = slice + (yy == 0 ? c.L - 1 : yy - 1) * c.L + xx;
    n.yp = slice + (yy == c.L - 1 ? 0 : yy + 1) * c.L + xx;
    const int tt = dag ? (t == 0 ? c.Nt - 1 : t - 1) : (t == c.Nt - 1 ? 0 : t + 1);
    n.tn = tt * c.LL + (s - slice);
    n.wrap_sign = dag ? (t == 0) : (t == c.Nt - 1);
    return n;
}

template <typename R>
__device__ __forceinline__ void phis(const BChainDev& c, int s, R& p1, R& p2, R& p3);
template <> __device__ __forceinline__ void phis<float>(const BChainDev& c, int s, float& p1, float& p2, float& p3) {
    p1 = __ldg(c.phi32 + s); p2 = __ldg(c.phi32 + c.V + s); p3 = __ldg(c.phi32 + 2 * c.V + s);
}
template <> __device__ __forceinline__ void phis<double>(const BChainDev& c, int s, double& p1, double& p2, double& p3) {
    p1 = __ldg(c.phi64 + s); p2 = __ldg(c.phi64 + c.V + s); p3 = __ldg(c.phi64 + 2 * c.V + s);
}
__device__ __forceinline__ float eta_of(const BChainDev& c, int s) {
    int xx, yy, t;
    site_coords(c, s, xx, yy, t);
    return ((xx + yy) & 1) ? -1.f : 1.f;
}

template <typename R> __device__ __forceinline__ Site<R> axpy_site(R a, const Site<R>& x, const Site<R>& y) {
    Site<R> o;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        o.c[q].x = fma(a, x.c[q].x, y.c[q].x);
        o.c[q].y = fma(a, x.c[q].y, y.c[q].y);
    }
    return o;
}
template <typename R> __device__ __forceinline__ double norm2_site(const Site<R>& v) {
    double n = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) n += (double)v.c[q].x * v.c[q].x + (double)v.c[q].y * v.c[q].y;
    return n;
}

// block sum of v written to part[tile * 2 + j] by thread 0
__device__ __forceinline__ void tile_sum(double v, double* part, int tile, int j, double* red) {
    const double s = block_sum(v, red);
    if (threadIdx.x == 0) part[tile * 2 + j] = s;
}

// Sum of a pair's tile partials by the calling warp (lane l takes tiles l, l + 32, ..., then a fixed
// shuffle tree): every lane gets the result; the order is fixed, so the sum is reproducible.
__device__ __forceinline__ double pair_sum(const BatchArgs& a, int p, int j) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int t = a.pair_t0[p] + lane; t < a.pair_t0[p + 1]; t += 32) s += ldcg_dbl(a.part + t * 2 + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}
__device__ __forceinline__ int active_of(const BatchArgs& a, int p) { return ldcg_int(&a.sc[p].active); }

// Three blocks per SM (80 registers; the FP64 reliable-update phases spill a little): the phases
// wait on L2 neighbour loads, and 24 resident warps per SM ran the 64-chain trajectory in 0.88 s
// against 0.96 s with 16 (two blocks, 90 registers), 0.90 s with 32 and 0.92 s with 40 (spilling).
__global__ void __launch_bounds__(kBThreads, 3) k_batched_cg(BatchArgs a) {
    __shared__ double red[kBThreads / 32];
    const int G = gridDim.x;
    const int K = a.K;
    auto pair_base = [&](const BChainDev& c, int k) { return c.off + (int64_t)k * c.V; };
    bool ok = true;
    bool never = a.test_timeout != 0;

    // ---- start: r64 = b - A x64 (or b for a zero start), r32, x32 = 0, p = 0, norms ----------------
    if (a.use_x0) {
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Nbr n = neighbours(c, s, true);
                double p1, p2, p3;
                phis<double>(c, s, p1, p2, p3);
                const Site<double>* xv = a.x64 + base;
                Site<double> o = site_op<double>(a.cf64, ldcg_site(xv + n.c), ldcg_site(xv + n.xm), ldcg_site(xv + n.xp),
                                                 ldcg_site(xv + n.ym), ldcg_site(xv + n.yp), ldcg_site(xv + n.tn),
                                                 n.wrap_sign ? -1.0 : 1.0, p1, p2, p3, (double)eta_of(c, s));
                store_site(a.t64 + base + s, o);
            }
        }
        ok = grid_sync(a, never);
        never = false;
        if (!ok) return;
    }
    for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
        const BTile tl = a.tiles[ti];
        const BChainDev& c = a.ch[tl.chain];
        const int64_t base = pair_base(c, tl.pair - tl.chain * K);
        double b2 = 0.0, r2 = 0.0;
        for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
            const Site<double> bb = load_site(a.b + base + s);   // input, read-only
            Site<double> r = bb;
            if (a.use_x0) {
                const Nbr n = neighbours(c, s, false);
                double p1, p2, p3;
                phis<double>(c, s, p1, p2, p3);
                const Site<double>* tv = a.t64 + base;
                const Site<double> q = site_op<double>(a.cf64, ldcg_site(tv + n.c), ldcg_site(tv + n.xm),
                                                       ldcg_site(tv + n.xp), ldcg_site(tv + n.ym), ldcg_site(tv + n.yp),
                                                       ldcg_site(tv + n.tn), n.wrap_sign ? -1.0 : 1.0, p1, p2, p3,
                                                       (double)eta_of(c, s));
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    r.c[q4].x -= q.c[q4].x;
                    r.c[q4].y -= q.c[q4].y;
                }
            } else {
                store_site(a.x64 + base + s, Site<double>{});
                store_site(a.t64 + base + s, Site<double>{});   // D^dagger x of the zero start
            }
            store_site(a.r64 + base + s, r);
            Site<float> r32, z{};
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) r32.c[q4] = make_float2((float)r.c[q4].x, (float)r.c[q4].y);
            store_site(a.r32 + base + s, r32);
            store_site(a.x32 + base + s, z);
            store_site(a.pA + base + s, z);
            b2 += norm2_site(bb);
            r2 += norm2_site(r);
        }
        tile_sum(b2, a.part, ti, 0, red);
        tile_sum(r2, a.part, ti, 1, red);
    }
    if (!(ok = grid_sync(a, never))) return;
    never = false;
    for (int p = blockIdx.x; p < a.npairs; p += G) {
        if (threadIdx.x < 32) {
            BScal s{};
            s.b2 = pair_sum(a, p, 0);
            s.r2 = pair_sum(a, p, 1);
            if (threadIdx.x != 0) continue;
            s.r2_max = s.r2;
            s.r2true = s.r2;
            s.rr = s.r2;
            s.nonfinite = (isfinite(s.b2) && isfinite(s.r2)) ? 0 : 1;
            s.active = (!s.nonfinite && s.b2 > 0.0 && s.r2 > a.tol2 * s.b2) ? 1 : 0;
            a.sc[p] = s;
            if (s.active) atomicAdd(a.nactive, 1);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.flags[1] = 0;
        a.iters_out[0] = 0;
        a.iters_out[1] = 0;
    }
    if (!(ok = grid_sync(a, false))) return;

    Site<float>* pold = a.pA;
    Site<float>* pnew = a.pB;
    for (int it = 0; it < a.maxit; ++it) {
        if (ldcg_int(a.nactive) <= 0) break;   // every pair has converged (or stopped)
        // ---- I: p = r + beta p_old, t_ = D^dagger p, ||t_||^2 ----
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            if (!active_of(a, tl.pair)) continue;
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            const float beta = (float)ldcg_dbl(&a.sc[tl.pair].beta);
            const Site<float>* rv = a.r32 + base;
            const Site<float>* pv = pold + base;
            auto pp = [&](int j) { return axpy_site<float>(beta, ldcg_site(pv + j), ldcg_site(rv + j)); };
            double n2 = 0.0;
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Nbr n = neighbours(c, s, true);
                float p1, p2, p3;
                phis<float>(c, s, p1, p2, p3);
                const Site<float> pc = pp(n.c);
                const Site<float> t = site_op<float>(a.cf32, pc, pp(n.xm), pp(n.xp), pp(n.ym), pp(n.yp), pp(n.tn),
                                                     n.wrap_sign ? -1.f : 1.f, p1, p2, p3, eta_of(c, s));
                store_site(pnew + base + s, pc);
                store_site(a.t32 + base + s, t);
                n2 += norm2_site(t);
            }
            tile_sum(n2, a.part, ti, 0, red);
        }
        if (!(ok = grid_sync(a, false))) return;
        // ---- II + III: alpha of the tile's pair, q = D t_, x += alpha p, r -= alpha q, ||r||^2 ----
        __shared__ double s_alpha;
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            if (!active_of(a, tl.pair)) continue;
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            // every block holding a tile of the pair forms the same alpha (same partials, same order)
            if (threadIdx.x < 32) {
                const double pAp = pair_sum(a, tl.pair, 0);
                if (threadIdx.x == 0) {
                    s_alpha = (pAp > 0.0 && isfinite(pAp)) ? ldcg_dbl(&a.sc[tl.pair].rr) / pAp : 0.0;
                    if (!isfinite(pAp)) a.sc[tl.pair].nonfinite = 1;
                }
            }
            __syncthreads();
            const float alpha = (float)s_alpha;
            const Site<float>* tv = a.t32 + base;
            double r2 = 0.0;
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Nbr n = neighbours(c, s, false);
                float p1, p2, p3;
                phis<float>(c, s, p1, p2, p3);
                const Site<float> q = site_op<float>(a.cf32, ldcg_site(tv + n.c), ldcg_site(tv + n.xm),
                                                     ldcg_site(tv + n.xp), ldcg_site(tv + n.ym), ldcg_site(tv + n.yp),
                                                     ldcg_site(tv + n.tn), n.wrap_sign ? -1.f : 1.f, p1, p2, p3,
                                                     eta_of(c, s));
                const Site<float> x = axpy_site<float>(alpha, ldcg_site(pnew + base + s), ldcg_site(a.x32 + base + s));
                const Site<float> r = axpy_site<float>(-alpha, q, ldcg_site(a.r32 + base + s));
                store_site(a.x32 + base + s, x);
                store_site(a.r32 + base + s, r);
                r2 += norm2_site(r);
            }
            tile_sum(r2, a.part, ti, 1, red);
        }
        if (!(ok = grid_sync(a, false))) return;
        // ---- IV: beta, convergence, reliable-update request ----
        for (int p = blockIdx.x; p < a.npairs; p += G) {
            if (threadIdx.x < 32 && active_of(a, p)) {
                BScal& s = a.sc[p];
                const double r2 = pair_sum(a, p, 1);
                if (threadIdx.x != 0) continue;
                const double rr = ldcg_dbl(&s.rr);
                s.beta = rr > 0.0 ? r2 / rr : 0.0;
                s.rr = r2;
                s.r2 = r2;
                const int iters = ldcg_int(&s.iters) + 1;
                s.iters = iters;
                if (!isfinite(r2)) {
                    s.nonfinite = 1;
                    s.active = 0;
                    atomicSub(a.nactive, 1);
                } else if (r2 <= a.tol2 * ldcg_dbl(&s.b2) || r2 < a.delta2 * ldcg_dbl(&s.r2_max)) {
                    s.need_ru = 1;
                    atomicOr(a.flags + 1, 1);
                }
                atomicMax(a.iters_out, iters);
            }
        }
        { Site<float>* tmp = pold; pold = pnew; pnew = tmp; }
        if (!(ok = grid_sync(a, false))) return;
        if (!ldcg_int(a.flags + 1) && it + 1 < a.maxit) continue;
        // ---- reliable update (every pair with need_ru; at maxit every active pair) ----
        const bool last = it + 1 >= a.maxit;
        auto wants = [&](int p) { return active_of(a, p) && (ldcg_int(&a.sc[p].need_ru) || last); };
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            if (!wants(tl.pair)) continue;
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Site<float> lo = ldcg_site(a.x32 + base + s);
                Site<double> hi = ldcg_site(a.x64 + base + s);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    hi.c[q4].x += (double)lo.c[q4].x;
                    hi.c[q4].y += (double)lo.c[q4].y;
                }
                store_site(a.x64 + base + s, hi);
                store_site(a.x32 + base + s, Site<float>{});
            }
        }
        if (!(ok = grid_sync(a, false))) return;
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            if (!wants(tl.pair)) continue;
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            const Site<double>* xv = a.x64 + base;
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Nbr n = neighbours(c, s, true);
                double p1, p2, p3;
                phis<double>(c, s, p1, p2, p3);
                store_site(a.t64 + base + s,
                           site_op<double>(a.cf64, ldcg_site(xv + n.c), ldcg_site(xv + n.xm), ldcg_site(xv + n.xp),
                                           ldcg_site(xv + n.ym), ldcg_site(xv + n.yp), ldcg_site(xv + n.tn),
                                           n.wrap_sign ? -1.0 : 1.0, p1, p2, p3, (double)eta_of(c, s)));
            }
        }
        if (!(ok = grid_sync(a, false))) return;
        for (int ti = blockIdx.x; ti < a.ntiles; ti += G) {
            const BTile tl = a.tiles[ti];
            if (!wants(tl.pair)) continue;
            const BChainDev& c = a.ch[tl.chain];
            const int64_t base = pair_base(c, tl.pair - tl.chain * K);
            const Site<double>* tv = a.t64 + base;
            double r2 = 0.0;
            for (int s = tl.s0 + threadIdx.x; s < tl.s1; s += blockDim.x) {
                const Nbr n = neighbours(c, s, false);
                double p1, p2, p3;
                phis<double>(c, s, p1, p2, p3);
                const Site<double> q = site_op<double>(a.cf64, ldcg_site(tv + n.c), ldcg_site(tv + n.xm),
                                                       ldcg_site(tv + n.xp), ldcg_site(tv + n.ym), ldcg_site(tv + n.yp),
                                                       ldcg_site(tv + n.tn), n.wrap_sign ? -1.0 : 1.0, p1, p2, p3,
                                                       (double)eta_of(c, s));
                Site<double> r = load_site(a.b + base + s);
                Site<float> r32;
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    r.c[q4].x -= q.c[q4].x;
                    r.c[q4].y -= q.c[q4].y;
                    r32.c[q4] = make_float2((float)r.c[q4].x, (float)r.c[q4].y);
                }
                store_site(a.r64 + base + s, r);
                store_site(a.r32 + base + s, r32);
                r2 += norm2_site(r);
            }
            tile_sum(r2, a.part, ti, 1, red);
        }
        if (!(ok = grid_sync(a, false))) return;
        for (int p = blockIdx.x; p < a.npairs; p += G) {
            if (threadIdx.x < 32 && wants(p)) {
                BScal& s = a.sc[p];
                const double r2 = pair_sum(a, p, 1);
                if (threadIdx.x != 0) continue;
                s.r2true = r2;
                s.need_ru = 0;
                if (!isfinite(r2)) {
                    s.nonfinite = 1;
                    s.active = 0;
                    atomicSub(a.nactive, 1);
                } else if (r2 <= a.tol2 * ldcg_dbl(&s.b2)) {
                    s.active = 0;
                    atomicSub(a.nactive, 1);
                } else {
                    s.r2 = r2;
                    s.r2_max = r2;
                    s.rr = r2;
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.flags[1] = 0;
            a.iters_out[1] += 1;
        }
        if (!(ok = grid_sync(a, false))) return;
    }
}

__global__ void k_phi_to32_b(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---- host ----------------------------------------------------------------------------------------
void batch_free(hmc_ctx* ctx) {
    BatchWork& w = ctx->batch;
    void* ps[] = {w.tiles, w.pair_t0, w.sc, w.part, w.hist, w.hist_ru};
    for (void* p : ps)
        if (p) cudaFree(p);
    w.tiles = nullptr; w.pair_t0 = nullptr; w.sc = nullptr; w.part = nullptr; w.hist = nullptr; w.hist_ru = nullptr;
    w.K = 0;
    w.kcap = 0;
}

// Statistics of one pair after a solve.
struct BStat {
    double r2true, b2;
    int iters, flags;   // flags: 1 still active (not converged), 2 non-finite
};

// hist[slot][pair] from the solver scalars; hist_ru[slot] = reliable updates; hist_ru[HMC_MAX_SOLVES]
// collects the failure flags of every solve of the trajectory (also those past the last slot).
__global__ void k_batch_record(const BScal* __restrict__ sc, int npairs, const int* __restrict__ iters,
                               BStat* __restrict__ hist, int* __restrict__ hist_ru, int slot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    const BScal& s = sc[i];
    const int f = (s.active ? 1 : 0) | (s.nonfinite ? 2 : 0);
    if (f) atomicOr(hist_ru + HMC_MAX_SOLVES, f);
    if (slot >= HMC_MAX_SOLVES) return;
    hist[(int64_t)slot * npairs + i] = BStat{s.r2true, s.b2, s.iters, f};
    if (i == 0) hist_ru[slot] = iters[1];
}

int batch_alloc(hmc_ctx* ctx) {
    BatchWork& w = ctx->batch;
    const int nc = (int)ctx->chains.size(), K = ctx->kmax;
    int64_t nt = 0;
    for (int c = 0; c < nc; ++c) nt += (ctx->chains[c].lat.V + kTile - 1) / kTile;
    nt *= K;
    if (nt > (int64_t)1 << 30) return fail(ctx, HMC_ERR_ARG, "hmc_init: too many batched tiles");
    HMC_CUDA(ctx, cudaMalloc(&w.tiles, nt * sizeof(BTile)));
    HMC_CUDA(ctx, cudaMalloc((void**)&w.pair_t0, ((size_t)nc * K + 1) * sizeof(int)));
    HMC_CUDA(ctx, cudaMalloc(&w.sc, (size_t)nc * K * sizeof(BScal)));
    HMC_CUDA(ctx, cudaMalloc((void**)&w.part, nt * 2 * sizeof(double)));
    HMC_CUDA(ctx, cudaMalloc(&w.hist, (size_t)HMC_MAX_SOLVES * nc * K * sizeof(BStat)));
    HMC_CUDA(ctx, cudaMalloc((void**)&w.hist_ru, (HMC_MAX_SOLVES + 1) * sizeof(int)));
    w.kcap = K;
    w.ntiles_cap = (int)nt;
    w.K = 0;
    w.hch.resize(nc);
    return HMC_OK;
}

// Tile table for K right-hand sides (rebuilt only when K changes; synchronous copies into the
// buffers batch_alloc made).
static int batch_setup(hmc_ctx* ctx, int K) {
    BatchWork& w = ctx->batch;
    if (w.K == K) return HMC_OK;
    if (K < 1 || K > w.kcap) return fail(ctx, HMC_ERR_ARG, "batched solve: nrhs must be in [1, nrhs_max]");
    const int nc = (int)ctx->chains.size();
    std::vector<BTile> tiles;
    std::vector<int> pt0;
    for (int c = 0; c < nc; ++c) {
        const int V = (int)ctx->chains[c].lat.V;
        for (int k = 0; k < K; ++k) {
            pt0.push_back((int)tiles.size());
            for (int s0 = 0; s0 < V; s0 += kTile) tiles.push_back(BTile{c * K + k, c, s0, std::min(V, s0 + kTile)});
        }
    }
    pt0.push_back((int)tiles.size());
    HMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the tables may be in use by earlier work
    HMC_CUDA(ctx, cudaMemcpy(w.tiles, tiles.data(), tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice));
    HMC_CUDA(ctx, cudaMemcpy(w.pair_t0, pt0.data(), pt0.size() * sizeof(int), cudaMemcpyHostToDevice));
    w.ntiles = (int)tiles.size();
    w.K = K;
    int bps = 0;
    HMC_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_batched_cg, kBThreads, 0));
    if (bps < 1) return fail(ctx, HMC_ERR_CUDA, "batched solve: kernel does not fit on an SM");
    w.grid = std::min(ctx->num_sms * bps, w.ntiles);
    return HMC_OK;
}

int batched_begin(hmc_ctx* ctx, int K, const double* const* phi) {
    BatchWork& w = ctx->batch;
    int rc;
    if ((rc = batch_setup(ctx, K))) return rc;
    const int nc = (int)ctx->chains.size();
    for (int c = 0; c < nc; ++c) {
        const Lat& lat = ctx->chains[c].lat;
        BChainDev d{};
        d.L = lat.L;
        d.Nt = lat.Nt;
        d.LL = lat.L * lat.L;
        d.invL = 1.0f / (float)lat.L;
        d.invLL = 1.0f / (float)(lat.L * lat.L);
        d.V = lat.V;
        d.off = ctx->batch_off[c] * K;
        d.phi64 = phi[c];
        d.phi32 = ctx->batch_phi32 + 3 * ctx->batch_off[c];
        w.hch[c] = d;
    }
    HMC_CUDA(ctx, cudaMemcpyAsync(w.ch, w.hch.data(), nc * sizeof(BChainDev), cudaMemcpyHostToDevice, ctx->stream));
    HMC_CUDA(ctx, cudaMemsetAsync(w.hist_ru + HMC_MAX_SOLVES, 0, sizeof(int), ctx->stream));
    return HMC_OK;
}

int batched_solve(hmc_ctx* ctx, int K, const double2* b, double2* x, bool use_x0, double tol, int maxit, int slot) {
    BatchWork& w = ctx->batch;
    if (w.K != K) return fail(ctx, HMC_ERR_STATE, "batched solve: batched_begin was not called for this nrhs");
    const int nc = (int)ctx->chains.size();
    for (int c = 0; c < nc; ++c) {
        const BChainDev& d = w.hch[c];
        k_phi_to32_b<<<(unsigned)((3 * d.V + 255) / 256), 256, 0, ctx->stream>>>(d.phi64, const_cast<float*>(d.phi32),
                                                                                 3 * d.V);
        HMC_LAUNCH(ctx, "k_phi_to32");
    }
    BatchArgs a{};
    a.nchains = nc;
    a.K = K;
    a.ntiles = w.ntiles;
    a.npairs = nc * K;
    a.ch = w.ch;
    a.tiles = reinterpret_cast<const BTile*>(w.tiles);
    a.pair_t0 = w.pair_t0;
    a.cf32 = make_coef<float>(ctx->p);
    a.cf64 = make_coef<double>(ctx->p);
    a.b = reinterpret_cast<const Site<double>*>(b);
    a.x64 = reinterpret_cast<Site<double>*>(x);
    a.r64 = reinterpret_cast<Site<double>*>(ctx->d_r64);
    a.t64 = reinterpret_cast<Site<double>*>(ctx->d_z64);
    a.x32 = reinterpret_cast<Site<float>*>(ctx->d_x32);
    a.r32 = reinterpret_cast<Site<float>*>(ctx->d_r32);
    a.pA = reinterpret_cast<Site<float>*>(ctx->d_p32);
    a.pB = reinterpret_cast<Site<float>*>(ctx->d_p32b);
    a.t32 = reinterpret_cast<Site<float>*>(ctx->d_q32);
    a.sc = reinterpret_cast<BScal*>(w.sc);
    a.part = w.part;
    a.bar = w.bar;
    a.flags = ctx->d_flags;
    a.nactive = w.iters + 2;
    a.iters_out = w.iters;
    a.tol2 = tol * tol;
    a.delta2 = 1e-6;
    a.maxit = maxit;
    a.use_x0 = use_x0 ? 1 : 0;
    a.test_timeout = ctx->p.test_wait_timeout;
    a.timeout_ns = ctx->p.wait_spin_limit > 0 ? (long long)ctx->p.wait_spin_limit * 1000LL : 2000000000LL;
    HMC_CUDA(ctx, cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), ctx->stream));
    HMC_CUDA(ctx, cudaMemsetAsync(w.iters, 0, 4 * sizeof(int), ctx->stream));
    // cooperative launch through the attribute form, which stream capture records as a
    // cooperative kernel node
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)w.grid);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HMC_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_batched_cg, a));
    HMC_LAUNCH(ctx, "k_batched_cg");
    k_batch_record<<<(unsigned)((nc * K + 127) / 128), 128, 0, ctx->stream>>>(
        reinterpret_cast<const BScal*>(w.sc), nc * K, w.iters, reinterpret_cast<BStat*>(w.hist), w.hist_ru, slot);
    HMC_LAUNCH(ctx, "k_batch_record");
    return HMC_OK;
}

int batched_collect(hmc_ctx* ctx, int K, int nsolves, int* iterations, double* worst_resid, int* reliable_updates) {
    BatchWork& w = ctx->batch;
    const int nc = (int)ctx->chains.size(), np = nc * K;
    const int kept = std::min(nsolves, HMC_MAX_SOLVES);
    std::vector<BStat> hs((size_t)kept * np);
    std::vector<int> hr(HMC_MAX_SOLVES + 1);
    if (kept > 0)
        HMC_CUDA(ctx, cudaMemcpyAsync(hs.data(), w.hist, hs.size() * sizeof(BStat), cudaMemcpyDeviceToHost, ctx->stream));
    HMC_CUDA(ctx, cudaMemcpyAsync(hr.data(), w.hist_ru, hr.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    int rc;
    if ((rc = check_device_flags(ctx))) return rc;   // synchronises
    for (int j = 0; j < kept; ++j) {
        for (int c = 0; c < nc; ++c) {
            double wr = 0.0;
            int it = 0;
            for (int k = 0; k < K; ++k) {
                const BStat& s = hs[(size_t)j * np + c * K + k];
                const double rel = s.b2 > 0.0 ? std::sqrt(s.r2true / s.b2) : 0.0;
                if (!(rel <= wr)) wr = rel;
                if (s.iters > it) it = s.iters;
            }
            iterations[(size_t)j * nc + c] = it;
            worst_resid[(size_t)j * nc + c] = wr;
        }
        reliable_updates[j] = hr[j];
    }
    const int f = hr[HMC_MAX_SOLVES];
    if (f & 2) return fail(ctx, HMC_ERR_NONFINITE, "batched solve: non-finite residual norm");
    if (f & 1) return fail(ctx, HMC_ERR_NOCONV, "batched solve: no convergence in " + std::to_string(ctx->p.cg_maxit) +
                                                   " iterations");
    return HMC_OK;
}

}  // namespace hmc
