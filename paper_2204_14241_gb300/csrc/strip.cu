// Fused complex64 y = A x = D (D^dagger x) (Eq. linsys) on full-height strips, for L a multiple
// of 16 up to 80.
//
// A pipeline is one strip of 16 columns x all L rows of one right-hand side, marched through a
// range of time slices. Because the strip spans the whole periodic y extent there is no halo in
// y; in x it stages two extra columns on each side (20 columns of x) and computes t_ = D^dagger x
// on one extra column on each side (18 columns). 16 x NSEG threads own a column segment of
// NY = L / NSEG consecutive rows each and walk down it with a three-row window in registers, so
// each row's y-neighbours cost one shared-memory site read instead of two; x(t-1) of its rows
// stays in registers for the time hop. 2 x NSEG side threads compute t_ on the two extra columns,
// each on the rows s, s + NSEG, ... so that the eight threads of a quarter warp read distinct
// bank groups.
//
// The blocks of one time chunk of a right-hand side run all its strips together, so a strip's
// halo columns are read while its neighbour strip has the same slices in L2. (An even split of all
// outputs over one block per SM put neighbouring strips at different slices and ran slower.)
//
// Per step t (x(t+1) landed in its TMA slot): barrier; then row by row, t_(t+1) = D^dagger x on
// the row into shared memory and y(t) = D t_ from t_(t) and the row's t_(t+1) still in registers,
// stored with one 32-byte store per site. The site arithmetic runs on packed (re, im) pairs with
// Blackwell's two-wide FP32 instructions (add/mul/fma .f32x2).
#include <cuda.h>

#include <cstring>
#include <functional>
#include <mutex>
#include <queue>
#include <vector>

#include "internal.h"

namespace hmc {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(u64 r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 swp2(u64 a) {   // (re, im) -> (im, re)
    float x, y;
    upk2(a, x, y);
    return pk2(y, x);
}

// One site, four complex components packed as (re, im) pairs; index c = alpha * 2 + spin.
struct P4 { u64 c[4]; };

// Coefficients of D with the real scalars broadcast to both halves of a pair.
struct CoefP {
    u64 d[2], hx[2], hy[2];
    float cpl;
};

static CoefP make_coef_p(const hmc_params& p) {
    CoefP c;
    auto bc = [](double v) {
        const float f = (float)v;
        u64 b;
        unsigned u;
        memcpy(&u, &f, 4);
        b = ((u64)u << 32) | u;
        return b;
    };
    for (int a = 0; a < 2; ++a) {
        c.d[a] = bc(-1.0 - p.dtau * p.mu[a]);
        c.hx[a] = bc(-p.dtau * p.t_h[a]);
        c.hy[a] = bc(-p.dtau * p.t_v[a]);
    }
    c.cpl = (float)(p.dtau * p.g);
    return c;
}

// One site of D v (time hop from v(t+1), ts = b(t)) or D^dagger v (from v(t-1), ts = b(t-1)):
//   out = d c + ts tn + hx (xm + xp) + hy (ym + yp) + cpl eta (phi.sigma) c[other band]
// with phi.sigma = [[p3, p1 - i p2], [p1 + i p2, -p3]] on spin and sigma^x swapping the bands.
__device__ __forceinline__ P4 site_op_p(const CoefP& cf, const P4& c, const P4& xm, const P4& xp, const P4& ym,
                                        const P4& yp, const P4& tn, u64 ts, float p1, float p2, float p3, float eta) {
    const float f = cf.cpl * eta;
    const float q1 = f * p1, q2 = f * p2, q3 = f * p3;
    const u64 Q1 = pk2(q1, q1), Q3 = pk2(q3, q3), NQ3 = pk2(-q3, -q3), Q2 = pk2(q2, -q2), NQ2 = pk2(-q2, q2);
    P4 o;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int i = a * 2 + s;
            const u64 u = add2(xm.c[i], xp.c[i]);
            const u64 v = add2(ym.c[i], yp.c[i]);
            u64 r = mul2(cf.d[a], c.c[i]);
            r = fma2(ts, tn.c[i], r);
            r = fma2(cf.hx[a], u, r);
            o.c[i] = fma2(cf.hy[a], v, r);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const u64 w0 = c.c[(1 - a) * 2], w1 = c.c[(1 - a) * 2 + 1];
        u64 r0 = fma2(Q3, w0, o.c[a * 2]);
        r0 = fma2(Q1, w1, r0);
        o.c[a * 2] = fma2(Q2, swp2(w1), r0);          // re += q2 w1.im, im -= q2 w1.re
        u64 r1 = fma2(Q1, w0, o.c[a * 2 + 1]);
        r1 = fma2(NQ2, swp2(w0), r1);                  // re -= q2 w0.im, im += q2 w0.re
        o.c[a * 2 + 1] = fma2(NQ3, w1, r1);
    }
    return o;
}

template <int L, int NY> struct StripShape {
    static constexpr int NSEG = L / NY;               // row segments
    static constexpr int NMAIN = 16 * NSEG;           // threads that own output columns
    static constexpr int NRING = 2 * NSEG;            // threads for the two side columns of t_
    static constexpr int NTHR = (NMAIN + NRING + 31) / 32 * 32;
    static constexpr int TC = 18;                     // columns of t_ computed
    // one staging slot (bytes): x of the 16 own columns [row][16 sites][32 B] (TMA 128-byte
    // swizzle), of the two columns left of the strip [row][2][32 B] and of the two right of it
    // [row][2][32 B] (64-byte swizzle); phi of the own columns [component][row][16]. Regions are
    // multiples of 1024 bytes.
    static constexpr int XMAIN = L * 16 * 32;
    static constexpr int XHALO = L * 2 * 32;
    static constexpr int PHI = 3 * L * 16 * 4;
    static constexpr int OFF_XL = XMAIN, OFF_XR = OFF_XL + XHALO, OFF_PHI = OFF_XR + XHALO;
    static constexpr int SLOT = OFF_PHI + PHI;
    static constexpr int TS = 2 * L * TC;             // 16-byte units per t_ slice [plane][row][18]
    static constexpr size_t smem = (size_t)2 * SLOT + (size_t)2 * TS * 16 + 1024;   // + alignment slack
    static_assert(L % 16 == 0 && L <= 80 && L % NY == 0, "strip kernel: L a multiple of 16 up to 80");
    static_assert(XMAIN % 1024 == 0 && XHALO % 1024 == 0 && PHI % 1024 == 0, "swizzled TMA regions 1024-byte aligned");
};

// Site `site` of a swizzled site-major region (16-byte units from `region`): unit u = 2 site + h
// of half h sits at u ^ ((u >> 3) & mask), the TMA swizzle of the region's box: mask 7 for the
// 128-byte swizzle of the 16 own columns (box rows of 4 sites), 3 for the 64-byte swizzle of the
// two side columns (box rows of 2 sites). A quarter warp's reads of one half of eight consecutive
// sites of a row, or of one side column on four consecutive rows of each side, hit eight distinct
// bank groups.
__device__ __forceinline__ P4 lds_site(const ulonglong2* region, int site, int lim, int mask) {
    if (!HMC_IN(site >= 0 && 2 * site + 1 < lim, kBndStripShared)) return P4{};
    const int u = (2 * site) ^ ((site >> 2) & mask);
    const ulonglong2 a = region[u], b = region[u ^ 1];
    P4 r;
    r.c[0] = a.x; r.c[1] = a.y; r.c[2] = b.x; r.c[3] = b.y;
    return r;
}

// Site i of a two-plane region starting at plane0 (plane stride pstride); lim bounds the 16-byte
// units readable from plane0 (checked in the bounds build only).
__device__ __forceinline__ P4 lds_p4(const ulonglong2* plane0, int pstride, int i, int lim) {
    if (!HMC_IN(i >= 0 && i + pstride < lim, kBndStripShared)) return P4{};
    const ulonglong2 a = plane0[i], b = plane0[pstride + i];
    P4 s;
    s.c[0] = a.x; s.c[1] = a.y; s.c[2] = b.x; s.c[3] = b.y;
    return s;
}
__device__ __forceinline__ void sts_p4(ulonglong2* plane0, int pstride, int i, const P4& s) {
    plane0[i] = make_ulonglong2(s.c[0], s.c[1]);
    plane0[pstride + i] = make_ulonglong2(s.c[2], s.c[3]);
}
__device__ __forceinline__ P4 ldg_p4(const Site<float>* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 a = __ldg(q), b = __ldg(q + 1);
    P4 s;
    s.c[0] = a.x; s.c[1] = a.y; s.c[2] = b.x; s.c[3] = b.y;
    return s;
}
// One 32-byte store per site (sites are 32-byte aligned).
__device__ __forceinline__ void stg_p4(Site<float>* p, const P4& s) {
    asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(s.c[0]), "l"(s.c[1]), "l"(s.c[2]),
                 "l"(s.c[3])
                 : "memory");
}

// ---- TMA and mbarrier primitives (inline PTX) ---------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase of parity `par` of the barrier: at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t par, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(bar), "r"(par) : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
// Bulk-tensor prefetch of a box into L2 (no shared memory, no barrier).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor maps of one launch: x viewed as [slice = k * Nt + t][y][x / 4][32 floats] for the own
// columns (box: 4 units of 4 sites x all rows, 128-byte swizzle) and as [slice][y][x / 2][16
// floats] for the side columns (box: 1 unit of 2 sites x all rows, 64-byte swizzle), phi as
// [component][t][y][x] (box: 16 columns x all rows x 3 components). Box rows of 128 and 64 bytes
// take a quarter and a half of the copy requests of whole-site (32-byte) rows, which the copy
// engine, not DRAM, was limited by.
struct StripMaps {
    CUtensorMap xmain, xhalo, phi;
};

// Grid: the blocks of StripSched sch (right-hand side k in sch.nch[k] time chunks, all strips of a
// chunk consecutive). part (if not null): part[k * nblk + c * (L / 16) + strip], nblk =
// sch.maxch * (L / 16), the partial sums of ||D^dagger x_k||^2 over the block's output sites (of
// ||A x_k||^2 in part_q with QN).
//
// Staging: two slots; slice x(ta + m) (and phi(ta + m) of the own columns) arrives by TMA in slot
// m & 1 on that slot's mbarrier, issued by thread 0 one step ahead. t_ lives in two slices.
// Step m: wait for slot m & 1; barrier (also the end of step m - 1); thread 0 issues slice m + 1
// into the other slot (read in step m - 1; phi of the rows a thread needs for y is kept in its
// registers from step m - 1); on each of its rows a thread writes t_(ta + m) = D^dagger x to the
// t_ slice that y(ta + m - 2) read one step earlier and computes y(ta + m - 1) = D t_ from
// t_(ta + m - 1) and the row's t_(ta + m) in registers. Nothing of t_(ta + m) is read before the
// next barrier, so one barrier per step.
// Waits are bounded (wait_limit polls): on a timeout the block drains the copy in flight, sets
// err[0] and returns. test_timeout makes the first wait target a barrier that is never armed.
// Slices prefetched into L2 ahead of the one loaded into the free slot: the two shared-memory
// slots keep one slice (66 KB at L = 80) in flight per SM, too little to cover the DRAM latency.
#ifndef STRIP_PREFETCH
#define STRIP_PREFETCH 3
#endif

template <int L, int NY, bool QN>
__global__ void __launch_bounds__(StripShape<L, NY>::NTHR, 1)
k_apply_A_strip(const __grid_constant__ StripMaps maps, Lat lat, CoefP cf, const __grid_constant__ StripSched sch,
                const float* __restrict__ phi, const Site<float>* __restrict__ x, Site<float>* __restrict__ y,
                double* __restrict__ part, double* __restrict__ part_q, const CgScalars* __restrict__ cgs,
                int* __restrict__ err, int wait_limit, int test_timeout) {
    using S = StripShape<L, NY>;
    constexpr int TC = S::TC, NSEG = S::NSEG;
    constexpr int nstrip = L / 16, LL = L * L;
    const int Nt = lat.Nt;
    const int64_t V = lat.V;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sbase = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    ulonglong2* tr = reinterpret_cast<ulonglong2*>(sbase + 2 * S::SLOT);   // 2 slices x [2 planes][L rows][18 columns]
    __shared__ __align__(8) uint64_t bars[3];   // two staging slots; the third is never armed (timeout test)
    __shared__ double red[S::NTHR / 32];

    const int tid = threadIdx.x;
    const bool own_y = tid < S::NMAIN;
    const bool has_t = tid < S::NMAIN + S::NRING;
    const bool side = has_t && !own_y;
    int tcol = 0, seg = 0;
    if (own_y) {
        tcol = 1 + (tid & 15);
        seg = tid >> 4;
    } else if (has_t) {
        const int r = tid - S::NMAIN;
        tcol = (r & 1) ? TC - 1 : 0;
        seg = r >> 1;
    }
    // row j of the thread: seg * NY + j (main), seg + NSEG * j (side)
    const int rstep = own_y ? 1 : NSEG;
    const int row0 = own_y ? seg * NY : seg;
    // staged x column of strip column j (j in [-2, 17]): its region (16-byte units from the slot),
    // the column within the region and the region's sites per row
    auto xcol_of = [&](int j, int& reg, int& col, int& rs) {
        if (j < 0) { reg = S::OFF_XL / 16; col = j + 2; rs = 2; }
        else if (j >= 16) { reg = S::OFF_XR / 16; col = j - 16; rs = 2; }
        else { reg = 0; col = j; rs = 16; }
    };
    int gc, oc, rc_, gl, ol, rl, gr, orr, rr;   // own column, left and right neighbour columns
    xcol_of(tcol - 1, gc, oc, rc_);
    xcol_of(tcol - 2, gl, ol, rl);
    xcol_of(tcol, gr, orr, rr);
    const int mc = gc == 0 ? 7 : 3, ml = gl == 0 ? 7 : 3, mr = gr == 0 ? 7 : 3;   // swizzle of each region
    constexpr int lim_slot = S::SLOT / 16;

    // this block's right-hand side k, time chunk c of nchk and strip sx (see StripSched)
    int b = blockIdx.x, k = 0, nchk = 1;
    for (int i = 0; i < sch.nrhs; ++i) {
        k = sch.order[i];
        nchk = sch.nch[k];
        if (b < nchk * nstrip) break;
        b -= nchk * nstrip;
    }
    const int c = b / nstrip, sx = b - c * nstrip;
    const bool active = !cgs || cgs[k].active;   // a converged right-hand side is left as it is
    const int ta = (int)((int64_t)c * Nt / nchk);
    const int tb = (int)((int64_t)(c + 1) * Nt / nchk);   // outputs y(ta .. tb-1); slices x(ta - 1 .. tb)

    const uint32_t bar0 = smem_u32(&bars[0]);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_init(bar0 + 16, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    constexpr uint32_t kSlotBytes = (uint32_t)S::SLOT;
    u64 acc = 0;   // (sum re^2, sum im^2) of t_ on the own output sites; with QN (sum |t_|^2, sum |y|^2)
    const int x0 = sx * 16;
    int gx = x0 - 1 + tcol;
    gx = gx < 0 ? gx + L : (gx >= L ? gx - L : gx);
    const Site<float>* xk = x + (int64_t)k * V;
    Site<float>* yk = y + (int64_t)k * V;
    // x columns x0 - 2, x0 - 1 and x0 + 16, x0 + 17 of the side boxes (thread 0 only)
    auto side_cols = [&](int& xl, int& xr) {
        xl = x0 - 2 < 0 ? x0 - 2 + L : x0 - 2;
        xr = x0 + 16 >= L ? x0 + 16 - L : x0 + 16;
    };
    auto issue = [&](int slot, int t) {   // thread 0 only
        const uint32_t bar = bar0 + 8 * slot;
        const uint32_t dst = smem_u32(sbase + slot * S::SLOT);
        const int sl = k * Nt + t;
        int xl, xr;
        side_cols(xl, xr);
        mbar_expect_tx(bar, kSlotBytes);
        tma_load_4d(dst, &maps.xmain, 0, x0 / 4, 0, sl, bar);
        tma_load_4d(dst + S::OFF_XL, &maps.xhalo, 0, xl / 2, 0, sl, bar);
        tma_load_4d(dst + S::OFF_XR, &maps.xhalo, 0, xr / 2, 0, sl, bar);
        tma_load_4d(dst + S::OFF_PHI, &maps.phi, x0, 0, t, 0, bar);
    };
    auto prefetch = [&](int t) {   // thread 0 only: the boxes of slice t into L2
        const int sl = k * Nt + t;
        int xl, xr;
        side_cols(xl, xr);
        tma_prefetch_4d(&maps.xmain, 0, x0 / 4, 0, sl);
        tma_prefetch_4d(&maps.xhalo, 0, xl / 2, 0, sl);
        tma_prefetch_4d(&maps.xhalo, 0, xr / 2, 0, sl);
        tma_prefetch_4d(&maps.phi, x0, 0, t, 0);
    };
    auto slice_of = [&](int m) { return ta + m >= Nt ? ta + m - Nt : ta + m; };
    const float eta0 = ((gx + row0) & 1) ? -1.f : 1.f;   // (-1)^(x+y) of row 0 of the thread

    // x(ta - 1) of the thread's rows; phi of slice ta on the side columns (not staged)
    P4 xprev[NY];
    float phk[NY][3];   // main: phi of the last t_ slice (the next y needs it); side: phi of the next t_ slice
    if (has_t && active) {
        const int tm = ta == 0 ? Nt - 1 : ta - 1;
#pragma unroll
        for (int j = 0; j < NY; ++j) {
            const int row = row0 + j * rstep;
            xprev[j] = P4{};
            if (HMC_IN(tm >= 0 && tm < Nt && row < L && gx >= 0 && gx < L, kBndStripGlobal))
                xprev[j] = ldg_p4(xk + (int64_t)tm * LL + row * L + gx);
            if (side) {
                const float* pp = phi + (int64_t)ta * LL + row * L + gx;
                phk[j][0] = __ldg(pp);
                phk[j][1] = __ldg(pp + V);
                phk[j][2] = __ldg(pp + 2 * V);
            }
        }
    }
    const int nsl = active ? tb - ta + 1 : 0;   // staged slices x(ta) .. x(tb)
    if (tid == 0 && nsl > 0) {
        issue(0, ta);
        for (int m = 1; m <= STRIP_PREFETCH && m < nsl; ++m) prefetch(slice_of(m));
    }
    for (int m = 0; m < nsl; ++m) {
        const int slot = m & 1;
        const uint32_t par = (uint32_t)((m >> 1) & 1);
        const int tn_slice = ta + m >= Nt ? ta + m - Nt : ta + m;   // slice of t_ computed now
        const bool ok = (test_timeout && m == 0) ? mbar_wait(bar0 + 16, 0, wait_limit)
                                                  : mbar_wait(bar0 + 8 * slot, par, wait_limit);
        if (__syncthreads_or(!ok)) {
            // drain the copy in flight into this slot before leaving (bounded as well)
            if (tid == 0) {
                if (!mbar_wait(bar0 + 8 * slot, par, wait_limit)) atomicOr(err, 2);
                atomicOr(err, 1);
            }
            __syncthreads();
            return;
        }
        if (tid == 0 && m + 1 < nsl) {
            fence_proxy_async();
            issue(slot ^ 1, slice_of(m + 1));
            if (m + 1 + STRIP_PREFETCH < nsl) prefetch(slice_of(m + 1 + STRIP_PREFETCH));
        }
        const ulonglong2* xb = reinterpret_cast<const ulonglong2*>(sbase + slot * S::SLOT);
        const float* phs = reinterpret_cast<const float*>(sbase + slot * S::SLOT + S::OFF_PHI);
        ulonglong2* tn = tr + slot * S::TS;                 // t_(tn_slice)
        const ulonglong2* tc = tr + (slot ^ 1) * S::TS;    // t_(tn_slice - 1)
        const u64 ts = tn_slice == 0 ? pk2(-1.f, -1.f) : pk2(1.f, 1.f);   // b(t - 1) of D^dagger
        const ulonglong2 *xc_r = xb + gc, *xl_r = xb + gl, *xr_r = xb + gr;
        if (own_y) {
            // Row by row down the column: t_(tn_slice) = D^dagger x on row j (into shared memory for
            // the neighbours), then y(t) = D t_ on row j at t = tn_slice - 1 from t_(t) of the
            // previous step and this row's t_(t + 1), still in registers; phi(t) of the row is kept
            // from the previous step.
            const int rup = row0 == 0 ? L - 1 : row0 - 1;
            const int rdn = row0 + NY == L ? 0 : row0 + NY;
            const bool do_y = m >= 1;
            const int t = tn_slice == 0 ? Nt - 1 : tn_slice - 1;
            const u64 tsy = t == Nt - 1 ? pk2(-1.f, -1.f) : pk2(1.f, 1.f);   // b(t) of D
            Site<float>* dst = yk + (int64_t)t * LL + row0 * L + gx;
            P4 up = lds_site(xc_r, rup * rc_ + oc, lim_slot - gc, mc);
            P4 cen = lds_site(xc_r, row0 * rc_ + oc, lim_slot - gc, mc);
            P4 tup, tcen;
            if (do_y) {
                tup = lds_p4(tc, L * TC, rup * TC + tcol, S::TS);
                tcen = lds_p4(tc, L * TC, row0 * TC + tcol, S::TS);
            }
#pragma unroll
            for (int j = 0; j < NY; ++j) {
                const int rd = j + 1 < NY ? row0 + j + 1 : rdn;
                const float eta = (j & 1) ? -eta0 : eta0;
                P4 tnew;
                {
                    const P4 dn = lds_site(xc_r, rd * rc_ + oc, lim_slot - gc, mc);
                    const P4 lf = lds_site(xl_r, (row0 + j) * rl + ol, lim_slot - gl, ml);
                    const P4 rt = lds_site(xr_r, (row0 + j) * rr + orr, lim_slot - gr, mr);
                    const float* qp = phs + (row0 + j) * 16 + (tcol - 1);
                    const float p1 = qp[0], p2 = qp[L * 16], p3 = qp[2 * L * 16];
                    tnew = site_op_p(cf, cen, lf, rt, up, dn, xprev[j], ts, p1, p2, p3, eta);
                    sts_p4(tn, L * TC, (row0 + j) * TC + tcol, tnew);
                    xprev[j] = cen;
                    up = cen;
                    cen = dn;
                    if (do_y) {
                        const P4 tdn = lds_p4(tc, L * TC, rd * TC + tcol, S::TS);
                        const P4 tlf = lds_p4(tc, L * TC, (row0 + j) * TC + tcol - 1, S::TS);
                        const P4 trt = lds_p4(tc, L * TC, (row0 + j) * TC + tcol + 1, S::TS);
                        const P4 ov = site_op_p(cf, tcen, tlf, trt, tup, tdn, tnew, tsy, phk[j][0], phk[j][1],
                                                phk[j][2], eta);
                        if (HMC_IN(t >= 0 && t < Nt && row0 + j < L && gx >= 0 && gx < L, kBndStripGlobal))
                            stg_p4(dst + j * L, ov);
                        if constexpr (QN) {
                            // acc = (sum |t_|^2, sum |y|^2): each site's two sums packed into one pair
                            u64 st = mul2(tcen.c[0], tcen.c[0]), sy = mul2(ov.c[0], ov.c[0]);
#pragma unroll
                            for (int qq = 1; qq < 4; ++qq) {
                                st = fma2(tcen.c[qq], tcen.c[qq], st);
                                sy = fma2(ov.c[qq], ov.c[qq], sy);
                            }
                            float t0, t1, y0, y1;
                            upk2(st, t0, t1);
                            upk2(sy, y0, y1);
                            acc = add2(acc, pk2(t0 + t1, y0 + y1));
                        } else {
#pragma unroll
                            for (int qq = 0; qq < 4; ++qq) acc = fma2(tcen.c[qq], tcen.c[qq], acc);
                        }
                        tup = tcen;
                        tcen = tdn;
                    }
                    phk[j][0] = p1;
                    phk[j][1] = p2;
                    phk[j][2] = p3;
                }
            }
        } else if (side) {
            // t_ on a side column, rows seg + NSEG j; phi prefetched one step ahead
#pragma unroll
            for (int j = 0; j < NY; ++j) {
                const int row = row0 + j * NSEG;
                const int ru = row == 0 ? L - 1 : row - 1, rd = row == L - 1 ? 0 : row + 1;
                const P4 cen = lds_site(xc_r, row * rc_ + oc, lim_slot - gc, mc);
                const P4 up = lds_site(xc_r, ru * rc_ + oc, lim_slot - gc, mc);
                const P4 dn = lds_site(xc_r, rd * rc_ + oc, lim_slot - gc, mc);
                const P4 lf = lds_site(xl_r, row * rl + ol, lim_slot - gl, ml);
                const P4 rt = lds_site(xr_r, row * rr + orr, lim_slot - gr, mr);
                const float eta = ((gx + row) & 1) ? -1.f : 1.f;
                const P4 ov = site_op_p(cf, cen, lf, rt, up, dn, xprev[j], ts, phk[j][0], phk[j][1], phk[j][2], eta);
                sts_p4(tn, L * TC, row * TC + tcol, ov);
                xprev[j] = cen;
            }
            if (m + 1 < nsl) {
                const int nx = tn_slice + 1 == Nt ? 0 : tn_slice + 1;
#pragma unroll
                for (int j = 0; j < NY; ++j) {
                    const float* pp = phi + (int64_t)nx * LL + (row0 + j * NSEG) * L + gx;
                    phk[j][0] = __ldg(pp);
                    phk[j][1] = __ldg(pp + V);
                    phk[j][2] = __ldg(pp + 2 * V);
                }
            }
        }
    }
    float a0, a1;
    upk2(acc, a0, a1);
    // partial sums: slot c * nstrip + sx of right-hand side k's maxch * nstrip; the last chunk's
    // blocks zero the slots of the chunks their right-hand side does not have
    const int64_t stride = (int64_t)sch.maxch * nstrip, slot_out = (int64_t)k * stride + c * nstrip + sx;
    if (part) {
        const double tot = block_sum(QN ? (double)a0 : (double)a0 + (double)a1, red);
        if (tid == 0) part[slot_out] = tot;
        if (c == nchk - 1)
            for (int cc = nchk + tid; cc < sch.maxch; cc += blockDim.x) part[(int64_t)k * stride + cc * nstrip + sx] = 0.0;
    }
    if (QN && part_q) {
        const double tot = block_sum((double)a1, red);
        if (tid == 0) part_q[slot_out] = tot;
        if (c == nchk - 1)
            for (int cc = nchk + tid; cc < sch.maxch; cc += blockDim.x) part_q[(int64_t)k * stride + cc * nstrip + sx] = 0.0;
    }
}

#ifndef STRIP_NY80
#define STRIP_NY80 4
#endif

bool strip_supported(const Lat& lat) {
    return lat.L % 16 == 0 && lat.L >= 16 && lat.L <= 80;
}

// Block schedule. A block stages C + 1 slices and computes C + 1 slices of t_ for C outputs, so it
// costs about C + 1.5 slice steps. Right-hand side k is cut into nch[k] equal time chunks, n or
// n + 1 of them; the right-hand sides with the longer chunks are launched first, so that blocks
// dealt to the SMs in launch order pair a long first block with a short second one instead of
// leaving SMs idle in a partial last wave (280 blocks on 152 SMs at 80x80x160 with 8 RHS cost 2 x
// 24.5 steps; 4 RHS in 7 chunks and 4 in 8 cost 46). The strips of one (k, chunk) are consecutive
// in the launch, so neighbouring strips read each other's halo columns from L2. The split is the
// one whose simulated greedy dealing over the resident block slots ends first.
static void strip_schedule(int Nt, int nrhs, int nstrip, int slots, StripSched* out) {
    double best = 1e300;
    int best_n = 1, best_m = 0;
    std::vector<double> cost;
    // chunk counts that fill at most 8 waves of the resident slots (more only adds block overhead)
    int64_t nmax = (int64_t)8 * slots / ((int64_t)nrhs * nstrip);
    if (nmax < 1) nmax = 1;
    if (nmax > Nt) nmax = Nt;
    for (int n = 1; n <= (int)nmax; ++n) {
        for (int m = 0; m <= nrhs; ++m) {
            if (m > 0 && n + 1 > Nt) break;
            cost.clear();
            for (int i = 0; i < nrhs; ++i) {
                const int nc = i < nrhs - m ? n : n + 1;
                for (int c = 0; c < nc; ++c) {
                    const double len = (double)((int64_t)(c + 1) * Nt / nc - (int64_t)c * Nt / nc) + 1.5;
                    for (int sx = 0; sx < nstrip; ++sx) cost.push_back(len);
                }
            }
            std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
            for (int i = 0; i < slots; ++i) free_at.push(0.0);
            double end = 0.0;
            for (double c : cost) {
                const double t = free_at.top() + c;
                free_at.pop();
                free_at.push(t);
                if (t > end) end = t;
            }
            if (end < best - 1e-9) { best = end; best_n = n; best_m = m; }
        }
    }
    out->maxch = best_m > 0 ? best_n + 1 : best_n;
    out->nblk = 0;
    for (int i = 0; i < nrhs; ++i) {
        out->order[i] = (unsigned char)i;
        out->nch[i] = (unsigned char)(i < nrhs - best_m ? best_n : best_n + 1);
        out->nblk += out->nch[i] * nstrip;
    }
}

static const StripSched* strip_sched(hmc_ctx* ctx, const Lat& lat, int nrhs, int slots) {
    for (const StripSched& s : ctx->strip_sched)
        if (s.L == lat.L && s.Nt == lat.Nt && s.nrhs == nrhs && s.slots == slots) return &s;
    StripSched s;
    s.L = lat.L;
    s.Nt = lat.Nt;
    s.nrhs = nrhs;
    s.slots = slots;
    strip_schedule(lat.Nt, nrhs, lat.L / 16, slots, &s);
    ctx->strip_sched.push_back(s);
    return &ctx->strip_sched.back();
}

// Host-only view of the block schedule (hmc.h): what a launch of the strip operator would run.
int strip_plan(int L, int Nt, int nrhs, int slots, int* nch, int* order, int* nblk) {
    if (L % 16 != 0 || L < 16 || L > 80 || Nt < 1 || nrhs < 1 || nrhs > 64 || slots < 1 || !nch || !order || !nblk)
        return fail(nullptr, HMC_ERR_ARG, "hmc_strip_plan: bad argument");
    StripSched s{};
    strip_schedule(Nt, nrhs, L / 16, slots, &s);
    for (int i = 0; i < nrhs; ++i) {
        nch[i] = s.nch[i];
        order[i] = s.order[i];
    }
    *nblk = s.nblk;
    return HMC_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link against
// the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn(hmc_ctx* ctx, int* rc) {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (err == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    *rc = fn ? HMC_OK : fail(ctx, HMC_ERR_CUDA, "apply_A: cuTensorMapEncodeTiled unavailable");
    return fn;
}

static int encode(hmc_ctx* ctx, EncodeTiledFn fn, CUtensorMap* m, const void* base, const cuuint64_t* dim,
                  const cuuint64_t* stride, const cuuint32_t* box, CUtensorMapSwizzle swz) {
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dim, stride, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, HMC_ERR_CUDA, "apply_A: tensor map rejected (" + std::to_string((int)r) + ")");
    return HMC_OK;
}

// The three tensor maps of a launch on x (all right-hand sides) and phi.
static int strip_maps(hmc_ctx* ctx, const Lat& lat, int nrhs, const float* phi, const void* x, StripMaps* m) {
    int rc;
    EncodeTiledFn fn = encode_fn(ctx, &rc);
    if (!fn) return rc;
    const cuuint64_t L = (cuuint64_t)lat.L;
    const cuuint64_t hdim[4] = {16, L / 2, L, (cuuint64_t)lat.Nt * (cuuint64_t)nrhs};   // 2 sites per unit
    const cuuint64_t hstr[3] = {64, 32 * L, 32 * L * L};
    const cuuint64_t wdim[4] = {32, L / 4, L, (cuuint64_t)lat.Nt * (cuuint64_t)nrhs};   // 4 sites per unit
    const cuuint64_t wstr[3] = {128, 32 * L, 32 * L * L};
    const cuuint32_t bmain[4] = {32, 4, (cuuint32_t)L, 1}, bhalo[4] = {16, 1, (cuuint32_t)L, 1};
    const cuuint64_t pdim[4] = {L, L, (cuuint64_t)lat.Nt, 3};
    const cuuint64_t pstr[3] = {4 * L, 4 * L * L, 4 * (cuuint64_t)lat.V};
    const cuuint32_t bphi[4] = {16, (cuuint32_t)L, 1, 3};
    if ((rc = encode(ctx, fn, &m->xmain, x, wdim, wstr, bmain, CU_TENSOR_MAP_SWIZZLE_128B))) return rc;
    if ((rc = encode(ctx, fn, &m->xhalo, x, hdim, hstr, bhalo, CU_TENSOR_MAP_SWIZZLE_64B))) return rc;
    return encode(ctx, fn, &m->phi, phi, pdim, pstr, bphi, CU_TENSOR_MAP_SWIZZLE_NONE);
}

template <int L, int NY>
static int go_strip(hmc_ctx* ctx, const Lat& lat, const float* phi, const Site<float>* x, Site<float>* y, int nrhs,
                    double* part, double* part_q, const CgScalars* cgs, int* nblk_out) {
    using S = StripShape<L, NY>;
    static PerDevice attr;
    uint64_t bit;
    if (attr.pending(&bit)) {
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A_strip<L, NY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)S::smem));
        HMC_CUDA(ctx, cudaFuncSetAttribute(k_apply_A_strip<L, NY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)S::smem));
        attr.mark(bit);
    }
    const int per_sm_smem = 228 * 1024;
    int bps = (int)(per_sm_smem / (S::smem + 1024));
    if (bps > 2048 / S::NTHR) bps = 2048 / S::NTHR;
    if (bps < 1) bps = 1;
    if (nrhs > 64) return fail(ctx, HMC_ERR_ARG, "apply_A: at most 64 right-hand sides per launch");
    const StripSched* sch = strip_sched(ctx, lat, nrhs, ctx->num_sms * bps);
    const int64_t nblk = (int64_t)sch->maxch * (L / 16);   // partial sums per right-hand side
    const int64_t cap = part_q ? ctx->part_cap / 2 : ctx->part_cap;   // part_q lives in the second half
    if ((part || part_q) && nblk * nrhs > cap) return fail(ctx, HMC_ERR_ARG, "apply_A: reduction buffer too small");
    StripMaps maps;
    int rc;
    if ((rc = strip_maps(ctx, lat, nrhs, phi, x, &maps))) return rc;
    const int wl = ctx->p.wait_spin_limit > 0 ? ctx->p.wait_spin_limit : (1 << 20);
    auto kern = part_q ? k_apply_A_strip<L, NY, true> : k_apply_A_strip<L, NY, false>;
    kern<<<(unsigned)sch->nblk, S::NTHR, S::smem, ctx->stream>>>(maps, lat, make_coef_p(ctx->p), *sch, phi, x, y, part,
                                                                 part_q, cgs, ctx->d_flags, wl, ctx->p.test_wait_timeout);
    HMC_LAUNCH(ctx, "k_apply_A_strip");
    if (nblk_out) *nblk_out = (int)nblk;
    return HMC_OK;
}

unsigned int bounds_take_strip() { return bounds_take_tu(); }

int launch_apply_A_strip(hmc_ctx* ctx, const Lat& lat, const float* phi, const float2* x, float2* y, int nrhs,
                         double* part, int* nblk_out, const CgScalars* cgs, double* part_q) {
    const Site<float>* xs = reinterpret_cast<const Site<float>*>(x);
    Site<float>* ys = reinterpret_cast<Site<float>*>(y);
    switch (lat.L) {
        case 16: return go_strip<16, 1>(ctx, lat, phi, xs, ys, nrhs, part, part_q, cgs, nblk_out);
        case 32: return go_strip<32, 2>(ctx, lat, phi, xs, ys, nrhs, part, part_q, cgs, nblk_out);
        case 48: return go_strip<48, 3>(ctx, lat, phi, xs, ys, nrhs, part, part_q, cgs, nblk_out);
        case 64: return go_strip<64, 4>(ctx, lat, phi, xs, ys, nrhs, part, part_q, cgs, nblk_out);
        case 80: return go_strip<80, STRIP_NY80>(ctx, lat, phi, xs, ys, nrhs, part, part_q, cgs, nblk_out);
        default: return fail(ctx, HMC_ERR_STATE, "apply_A: no strip kernel for this L");
    }
}

}  // namespace hmc

extern "C" int hmc_strip_plan(int L, int Nt, int nrhs, int slots, int* nch, int* order, int* nblk) {
    return hmc::strip_plan(L, Nt, nrhs, slots, nch, order, nblk);
}
