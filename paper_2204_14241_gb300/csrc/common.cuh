// Shared device definitions: complex helpers, lattice geometry, the per-site fermion
// stencil of Eq. (D_formula), and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hmc.h"

namespace hmc {

// ---- complex helpers --------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };
template <typename R> using cplx = typename CT<R>::T;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im) {
    C c; c.x = re; c.y = im; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {   // conj(a) * b
    C c; c.x = a.x * b.x + a.y * b.y; c.y = a.x * b.y - a.y * b.x; return c;
}

// Four complex components of one site, index c = alpha * 2 + spin.
template <typename R> struct Site { cplx<R> c[4]; };

template <typename R> __device__ __forceinline__ Site<R> load_site(const Site<R>* p) {
    Site<R> s;
    if constexpr (sizeof(R) == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
        float4 a = __ldg(q), b = __ldg(q + 1);
        s.c[0] = mk<float2>(a.x, a.y); s.c[1] = mk<float2>(a.z, a.w);
        s.c[2] = mk<float2>(b.x, b.y); s.c[3] = mk<float2>(b.z, b.w);
    } else {
        const double2* q = reinterpret_cast<const double2*>(p);
        s.c[0] = __ldg(q); s.c[1] = __ldg(q + 1); s.c[2] = __ldg(q + 2); s.c[3] = __ldg(q + 3);
    }
    return s;
}
template <typename R> __device__ __forceinline__ void store_site(Site<R>* p, const Site<R>& s) {
    if constexpr (sizeof(R) == 4) {
        float4* q = reinterpret_cast<float4*>(p);
        q[0] = make_float4(s.c[0].x, s.c[0].y, s.c[1].x, s.c[1].y);
        q[1] = make_float4(s.c[2].x, s.c[2].y, s.c[3].x, s.c[3].y);
    } else {
        double2* q = reinterpret_cast<double2*>(p);
        q[0] = s.c[0]; q[1] = s.c[1]; q[2] = s.c[2]; q[3] = s.c[3];
    }
}

// ---- lattice --------------------------------------------------------------------------
// Site index s = (t * L + y) * L + x.
struct Lat {
    int L, Nt;
    int64_t V;   // Nt * L * L
};

// Coefficients of D (Eq. D_formula) pre-multiplied by dtau.
template <typename R> struct Coef {
    R diag[2];   // -1 - dtau mu_alpha
    R hx[2];     // -dtau t_h[alpha]
    R hy[2];     // -dtau t_v[alpha]
    R cpl;       // dtau g
};

// b(t) = 1 - 2 delta_{t, Nt-1}: sign of the forward hop from slice t to t+1.
__device__ __forceinline__ int tnext(int t, int Nt) { return t + 1 == Nt ? 0 : t + 1; }
__device__ __forceinline__ int tprev(int t, int Nt) { return t == 0 ? Nt - 1 : t - 1; }
__device__ __forceinline__ int wrap_inc(int x, int L) { return x + 1 == L ? 0 : x + 1; }
__device__ __forceinline__ int wrap_dec(int x, int L) { return x == 0 ? L - 1 : x - 1; }

// One site of D v (DAG = false) or D^dagger v (DAG = true):
//   out = diag c + tsign * tn + hx (xm + xp) + hy (ym + yp) + cpl eta (phi.sigma) c[other band]
// tn is v at t+1 (D) or t-1 (D^dagger); tsign is b(t) for D and b(t-1) for D^dagger.
// The hopping is real symmetric and the on-site block Hermitian, so D and D^dagger differ
// only in the time hop.
template <typename R>
__device__ __forceinline__ Site<R> site_op(const Coef<R>& cf, const Site<R>& c, const Site<R>& xm,
                                           const Site<R>& xp, const Site<R>& ym, const Site<R>& yp,
                                           const Site<R>& tn, R tsign, R p1, R p2, R p3, R eta) {
    Site<R> o;
    const R f = cf.cpl * eta;
    const R q1 = f * p1, q2 = f * p2, q3 = f * p3;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const R d = cf.diag[a], hx = cf.hx[a], hy = cf.hy[a];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int i = a * 2 + s;
            R re = d * c.c[i].x + tsign * tn.c[i].x + hx * (xm.c[i].x + xp.c[i].x) + hy * (ym.c[i].x + yp.c[i].x);
            R im = d * c.c[i].y + tsign * tn.c[i].y + hx * (xm.c[i].y + xp.c[i].y) + hy * (ym.c[i].y + yp.c[i].y);
            o.c[i].x = re; o.c[i].y = im;
        }
        // sigma^x swaps the bands; phi.sigma = [[p3, p1 - i p2], [p1 + i p2, -p3]]
        const cplx<R> w0 = c.c[(1 - a) * 2], w1 = c.c[(1 - a) * 2 + 1];
        o.c[a * 2].x += q3 * w0.x + q1 * w1.x + q2 * w1.y;
        o.c[a * 2].y += q3 * w0.y + q1 * w1.y - q2 * w1.x;
        o.c[a * 2 + 1].x += q1 * w0.x - q2 * w0.y - q3 * w1.x;
        o.c[a * 2 + 1].y += q1 * w0.y + q2 * w0.x - q3 * w1.y;
    }
    return o;
}

// ---- reductions -------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0. smem needs blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* smem) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? smem[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// ---- index checks of the bounds build ----------------------------------------------------------
// Built with -DHMC_BOUNDS, each translation unit has a device error word; a failed check ORs its
// code into the word and the guarded access is skipped (never a trap). Otherwise the checks
// compile to nothing. hmc_bounds_status() (hmc.h) reads and clears the words.
#ifdef HMC_BOUNDS
static __device__ unsigned int hmc_bounds_word;
#define HMC_IN(cond, code) ((cond) ? true : (atomicOr(&hmc_bounds_word, (unsigned)(code)), false))
static inline unsigned int bounds_take_tu() {
    unsigned int w = 0, z = 0;
    if (cudaMemcpyFromSymbol(&w, hmc_bounds_word, sizeof(w)) != cudaSuccess) return 0x80000000u;
    cudaMemcpyToSymbol(hmc_bounds_word, &z, sizeof(z));
    return w;
}
#else
#define HMC_IN(cond, code) true
static inline unsigned int bounds_take_tu() { return 0; }
#endif
enum { kBndApplyD = 1, kBndForce = 2, kBndStripGlobal = 4, kBndStripShared = 8 };

// ---- asynchronous global -> shared copies (cp.async) ------------------------------------------
// 16-byte copies bypass L1 (.cg); both addresses 16-byte aligned. 4-byte copies go through L1.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace hmc
