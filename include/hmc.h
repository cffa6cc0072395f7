/*
 * hmc.h -- C ABI of the GB300 pseudofermion HMC library (libhmc.so) for the two-band
 * O(3) spin-fermion model of Lunts, Albergo and Lindsey, arXiv:2204.14241.
 *
 * Notation bridge. The paper calls the fermion matrix D(phi) (Eq. D_formula) and the
 * HMC mass matrix M. This ABI keeps the conventional names apply_M / apply_MdagM for
 * the FERMION matrix: "M" below is the paper's D, and apply_MdagM applies the paper's
 * Hermitian positive definite normal operator A = D D^dagger (Eq. linsys).
 *
 * Layouts (all field pointers are caller-owned, contiguous, device memory unless a
 * function says "host"):
 *   site index      s = (tau * L + y) * L + x            (x fastest; V = Nt * L * L)
 *   boson field     phi[a][s], a = 0, 1, 2               real, 3 * V entries
 *   fermion vector  v[k][s][alpha][spin]                 complex, interleaved re/im,
 *                   k < nrhs right-hand sides, alpha in {x-band, y-band}, 4 * V entries per k
 *   sigma-hat       sig[a][n_tau][m_y][m_x]              real, the metric's Fourier variances
 * The paper orders fermion indices (alpha, s, tau, x, y); the layout above is a
 * permutation of it with the four internal components of a site adjacent.
 *
 * Precision arguments: HMC_FP64 means phi is double and vectors are complex128
 * (double re, double im); HMC_FP32 means phi is float and vectors are complex64.
 *
 * Streams and synchronisation: every call is enqueued on the stream given to hmc_init
 * (0 = legacy default stream). Calls that return host scalars (S_pf, norms, stats,
 * trajectory results) synchronise that stream before returning; the others are
 * asynchronous. Workspace is allocated once in hmc_init; no call allocates afterwards.
 *
 * Errors: every function returns HMC_OK (0) or a positive code; hmc_last_error()
 * gives a one-line message. Invalid arguments never reach the GPU.
 */
#ifndef HMC_H
#define HMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum hmc_status {
    HMC_OK = 0,
    HMC_ERR_ARG = 1,        /* bad size, chain index, null pointer, or misaligned pointer */
    HMC_ERR_NOCONV = 2,     /* CG hit maxit; x holds the last iterate, stats the true residual */
    HMC_ERR_NONFINITE = 3,  /* NaN or Inf seen in a residual norm or an energy */
    HMC_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up (the work of that launch is incomplete) */
    HMC_ERR_CUDA = 5,       /* a CUDA runtime call failed; see hmc_last_error */
    HMC_ERR_STATE = 6       /* call not valid in the context's current state */
};

enum hmc_prec { HMC_FP64 = 0, HMC_FP32 = 1 };

/* Solver precision of a context: plain FP64 CG, or FP32 inner CG with FP64 reliable
 * updates (true residual and solution accumulated in FP64). */
enum hmc_solver_mode { HMC_SOLVER_FP64 = 0, HMC_SOLVER_MIXED = 1 };

enum hmc_noise { HMC_NOISE_EXPLICIT = 0, HMC_NOISE_PHILOX = 1 };

/* Model and solver parameters (Section "Sign-problem-free UV completion" and Section
 * "QMC path integral with fermions"; the lattice S_B is the forward-difference
 * discretisation of the paper's continuum boson action). */
typedef struct {
    int L;              /* spatial extent, even, >= 2 */
    int Nt;             /* time slices, >= 2 */
    double dtau;        /* Trotter step */
    double t_h[2];      /* nearest-neighbour hopping along x for bands x, y */
    double t_v[2];      /* nearest-neighbour hopping along y for bands x, y */
    double mu[2];       /* chemical potential per band */
    double g;           /* Yukawa coupling in D's on-site term dtau g (-1)^{x+y} phi.sigma sigma^x */
    double r;           /* boson mass term (r/2) phi^2 */
    double u;           /* quartic term (u/4) phi^4 */
    double c;           /* boson velocity: (1/c^2)(d_tau phi)^2 */
    int solver_mode;    /* hmc_solver_mode */
    int nrhs_max;       /* most pseudofermion right-hand sides per call, >= 1 */
    double cg_tol;      /* default relative true-residual tolerance ||b - A x|| / ||b|| */
    int cg_maxit;       /* default iteration cap */
    int initial_guess;  /* trajectory() force solves: 0 = zero start (default); m = 1 .. 5 =
                           chronological start from the polynomial extrapolation of degree m
                           through the trajectory's previous m + 1 solutions (m = 1:
                           2 X_n - X_{n-1}; 2: 3 X_n - 3 X_{n-1} + X_{n-2}; 3: 4 X_n - 6 X_{n-1}
                           + 4 X_{n-2} - X_{n-3}; ...; lower degree while fewer solutions exist),
                           m FP64 vectors of workspace. The same stopping test applies in every
                           case. */
    int autotune;       /* 0: tile shapes of the fused A kernel from a fixed rule (default; the
                           reduction order, hence every bit of the results, is reproducible);
                           1: on first use per (L, Nt, nrhs, precision) time the valid tile and
                           time-chunk shapes on the call's own buffers and keep the fastest */
    int wait_spin_limit;   /* polls of a device-side wait before it gives up (0: 1 << 20); a wait
                              that gives up makes the call return HMC_ERR_TIMEOUT */
    int test_wait_timeout; /* nonzero (tests only): the first device-side wait of every fused-A
                              launch (and the first grid barrier of a batched solve) targets a
                              barrier that nothing completes, so it always gives up */
    int batch_chains;   /* nonzero: trajectory() advances all chains together and every force
                           evaluation solves all (chain, RHS) pairs in one persistent cooperative
                           launch (mixed solver mode only; CG without the preconditioner; grid
                           barriers bounded by wait_spin_limit microseconds, default 2 s) */
    int batch_graph;    /* with batch_chains: the leapfrog part of a trajectory (every force
                           evaluation, kick and drift of all chains) runs as one CUDA graph,
                           captured on first use and replayed while n_leap, eps, the chains'
                           phi and sigma-hat buffers, nrhs and the solver settings stay the same;
                           its GPU time is then reported under the solve phase of
                           hmc_trajectory_stats (the per-phase split is not measured inside it) */
} hmc_params;

/* Per-chain lattice (batched chains of uneven sizes). Coupling constants other than r
 * are shared; L, Nt and r may differ per chain. */
typedef struct {
    int L, Nt;
    double r;
} hmc_chain;

/* Solver statistics (per call, over all right-hand sides). */
typedef struct {
    int iterations;          /* inner iterations of the slowest right-hand side */
    int reliable_updates;    /* FP64 true-residual recomputations (mixed mode) */
    int converged;           /* 1 if every right-hand side met the tolerance */
    double true_rel_resid;   /* max over RHS of ||b - A x|| / ||b||, evaluated in FP64 */
} hmc_cg_stats;

typedef struct hmc_ctx hmc_ctx;

/* Create a context for n_chains lattices. chains may be NULL, in which case every chain
 * uses p->L, p->Nt, p->r. cuda_stream is a cudaStream_t (or NULL for the default
 * stream). Allocates all device workspace on the device current at the call; every later
 * call on the context makes that device current for its duration and restores the caller's.
 * Errors: HMC_ERR_ARG, HMC_ERR_CUDA. */
int hmc_init(const hmc_params* p, int n_chains, const hmc_chain* chains, void* cuda_stream,
             hmc_ctx** out);
int hmc_destroy(hmc_ctx* ctx);
const char* hmc_last_error(const hmc_ctx* ctx);   /* ctx may be NULL (global last error) */

/* y = D x (dagger = 0) or y = D^dagger x (dagger = 1) for nrhs vectors -- Eq. (D_formula):
 * diagonal -1 - dtau mu_alpha, forward time hop with -1 at tau = Nt-1 (antiperiodic),
 * spatial hop -dtau t_alpha, on-site dtau g (-1)^{x+y} phi(tau,r).sigma (x) sigma^x.
 * phi: [3][V] in prec; x, y: [nrhs][V][4] complex in prec; x and y must not overlap. */
int apply_M(hmc_ctx* ctx, int chain, int prec, const void* phi, const void* x, void* y,
            int dagger, int nrhs);

/* y = A x = D (D^dagger x) (Eq. linsys), fused in one pass. If norm2 is not NULL it
 * receives (host, nrhs doubles) ||D^dagger x_k||^2 = x_k^dagger A x_k. */
int apply_MdagM(hmc_ctx* ctx, int chain, int prec, const void* phi, const void* x, void* y,
                int nrhs, double* norm2);

/* Allocation-free variant of apply_MdagM, for callers that must not allocate device memory
 * after start-up: code running under a memory pool or budget fixed in advance, an embedding
 * runtime that owns every allocation, or a caller that cannot use hmc_init because hmc_init
 * allocates its workspace. There is no counterpart in the paper; it computes exactly what
 * apply_MdagM computes (y = D D^dagger x and, if norm2 is not NULL, ||D^dagger x_k||^2 per
 * right-hand side into host memory) but takes the model parameters directly instead of a
 * context and keeps its reduction scratch in a fixed file-scope device array of 65536
 * doubles (512 KiB) plus 64 doubles of row sums, resident on every GPU that loads the library
 * until the process exits. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   p: model parameters (only dtau, t_h, t_v, mu and g are read); L, Nt: lattice; prec:
 *   HMC_FP64 or HMC_FP32 (as for apply_MdagM); phi, x, y: device, layouts as for apply_MdagM,
 *   16-byte aligned, the byte range of y disjoint from those of x and phi; 1 <= nrhs <= 65535
 *   (<= 64 when norm2 is requested); cuda_stream: cudaStream_t or NULL for the default stream.
 * It always runs the generic fused kernel (the one apply_MdagM uses for FP64 and for L not a
 * multiple of 16), never the complex64 strip kernel, so for complex64 with L a multiple of 16
 * it is slower than apply_MdagM; the results agree to rounding.
 * Set-up: the first call on each device (with that device current) looks up the device
 * address of the scratch array (cudaGetSymbolAddress); make that first call before any
 * stream capture. Every call on a device shares the one array and overwrites it, and each
 * slot it reads back is written earlier in the same call, so nothing needs clearing; calls
 * that can overlap on the GPU (other streams, other host threads) race on the array and
 * must be serialised by the caller. With norm2 the call synchronises cuda_stream.
 * Errors: HMC_ERR_ARG for bad arguments (including overlapping ranges), and when norm2 is
 * requested and nrhs times the number of tile blocks of the fused kernel exceeds the 65536
 * scratch slots (the message gives the count needed, its two factors and the limit);
 * HMC_ERR_CUDA for runtime failures. The message is available from hmc_last_error(NULL). */
int apply_MdagM_static(const hmc_params* p, int L, int Nt, int prec, const void* phi, const void* x, void* y,
                       int nrhs, double* norm2, void* cuda_stream);

/* y = P x with P = (K K^dagger)^{-1} = F~ P-hat F~^* (Eqs. Dsplit, twist, Kdiag, precon),
 * K the phi-independent part of D, applied with the twisted FFT. x, y: [nrhs][V][4] in prec
 * (device), owned by the caller; y may equal x (the complex64 spectrum between the passes is
 * kept in the context's workspace). Uses the context's stream; errors: HMC_ERR_ARG for a bad
 * chain, nrhs, pointer or precision. */
int apply_precond(hmc_ctx* ctx, int chain, int prec, const void* x, void* y, int nrhs);

/* Solve A x = b (Eq. linsys) by CG (precond = 0) or preconditioned CG (precond = 1),
 * zero initial guess, for nrhs right-hand sides at once. phi: [3][V] double; b, x:
 * complex128. Stops when the FP64 true residual of every RHS is <= tol ||b||.
 * tol <= 0 or maxit <= 0 select the context defaults. st may be NULL.
 * Returns HMC_ERR_NOCONV if maxit was reached (x then holds the last iterate). */
int cg_solve(hmc_ctx* ctx, int chain, const void* phi, const void* b, void* x, int nrhs,
             double tol, int maxit, int precond, hmc_cg_stats* st);

/* F = -dS/dphi for S = S_PF (+ S_B if include_boson) at phi (Eq. hamiltonseq), with
 * S_PF = sum_k varphi_k^dagger A^{-1} varphi_k (Eq. Z with pfs). The fermion part is
 * 2 dtau g (-1)^{x+y} Re[X^dagger (sigma^x (x) sigma^a) Y] per site, X = A^{-1} varphi,
 * Y = D^dagger X. phi: [3][V] double; phi_pf: [nrhs][V][4] complex128; F: [3][V] double
 * (overwritten). S_pf (host, may be NULL) receives 2 Re(varphi^dagger X) - ||Y||^2 summed
 * over RHS (equal to S_PF up to the square of the solver error); S_b (host, may be NULL)
 * receives S_B(phi). The solve uses the context tolerance and precond. */
int force(hmc_ctx* ctx, int chain, const void* phi, const void* phi_pf, int nrhs, void* F,
          double* S_pf, int include_boson, int precond, double* S_b, hmc_cg_stats* st);

/* Randomized diagonal estimator of Section "Fermionic observables": out = (1/K) sum_k
 * v_k . (O v_k) with O = F~^* D^{-1} F~ (the fermion Green's function in the twisted Fourier
 * basis of Eqs. twist, Kdiag), D^{-1} = D^dagger (D D^dagger)^{-1}, for K = nrhs probe vectors
 * with entries +-1 (E[v . O v] = diag(O)). The K solves are one multi-RHS CG (context tolerance;
 * precond as for cg_solve). phi: [3][V] double; v: [nrhs][V][4] complex128 (real parts +-1,
 * imaginary parts 0) in the twisted Fourier basis, site index (n_tau * L + m_y) * L + m_x;
 * out: [V][4] complex128 in the same basis. st may be NULL. */
int green_estimate(hmc_ctx* ctx, int chain, const void* phi, const void* v, int nrhs, void* out, int precond,
                   hmc_cg_stats* st);

/* Fourier-diagonal metric of Section "Online metric estimation" with the unitary DFT F
 * over (tau, y, x) per component and sigma-hat even in the wave vector:
 *   HMC_METRIC_MOMENTUM: out = F^{-1}(sigma^{-1/2} . F in)   (momentum draw from z = in)
 *   HMC_METRIC_VELOCITY: out = F^{-1}(sigma . F in)          (d phi / dt = M^{-1} pi)
 *   HMC_METRIC_KINETIC:  *scalar = (1/2) sum sigma |F in|^2  (out unused)
 *   HMC_METRIC_ACCUM:    out += |F in|^2                     (Eq. covest numerator)
 *   HMC_METRIC_MNORM:    *scalar = sum |F in|^2 / sigma      (in^T M in, M = Sigma^{-1}: the squared
 *                                                             jump distance of Eq. ESJD; out unused)
 * in, out: [3][V] double; sig: [3][V] double; scalar: host. */
enum hmc_metric_op { HMC_METRIC_MOMENTUM = 0, HMC_METRIC_VELOCITY = 1, HMC_METRIC_KINETIC = 2,
                     HMC_METRIC_ACCUM = 3, HMC_METRIC_MNORM = 4 };
int metric_apply(hmc_ctx* ctx, int chain, int op, const void* sig, const void* in, void* out,
                 double* scalar);

/* Inputs of one HMC update of every chain (Section "HMC": heatbath varphi = D chi,
 * pi ~ N(0, M), leapfrog, Metropolis). Arrays of device pointers have n_chains entries
 * and are themselves host arrays. */
typedef struct {
    void** phi;              /* [n_chains] device double [3][V]; replaced by the new state */
    const void** sigma_hat;  /* [n_chains] device double [3][V] */
    double eps;              /* leapfrog step */
    int n_leap;              /* leapfrog steps (n_leap + 1 force evaluations) */
    int nrhs;                /* pseudofermion right-hand sides per chain */
    int precond;             /* 1: preconditioned CG in every force evaluation */
    int noise;               /* hmc_noise */
    const void** chi;        /* EXPLICIT: [n_chains] device complex128 [nrhs][V][4], std complex normal */
    const void** z;          /* EXPLICIT: [n_chains] device double [3][V], N(0, 1) */
    const double* u;         /* EXPLICIT: [n_chains] host uniforms in [0, 1) */
    uint64_t seed;           /* PHILOX: key */
    uint64_t counter;        /* PHILOX: trajectory counter (distinct per trajectory) */
} hmc_traj_in;

/* Per-chain results, host arrays of n_chains entries (any may be NULL). energies holds
 * 6 doubles per chain: kinetic, S_B, S_PF at the start, then the same at the end. */
typedef struct {
    double* dH;
    int* accepted;
    double* energies;
    int* cg_iterations;      /* total inner CG iterations over the trajectory */
    double* max_true_resid;  /* worst final true relative residual of any solve */
    double* jump2;           /* (phi' - phi)^T M (phi' - phi) of the proposal, accepted or not */
} hmc_traj_out;

/* One HMC update of every chain. Returns HMC_ERR_NOCONV / HMC_ERR_NONFINITE if a solve
 * failed or an energy is not finite (phi is then restored to its input value). */
int trajectory(hmc_ctx* ctx, const hmc_traj_in* in, hmc_traj_out* out);

/* Per-solve and per-phase record of a chain's last trajectory (tracing, per-trajectory logs).
 * Phases (GPU time from CUDA events on the context's stream, milliseconds):
 *   phase_ms[0] the force solves (CG/PCG with reliable updates and chronological starts),
 *   phase_ms[1] the force kernel (D^dagger X contraction and boson force) and action reductions,
 *   phase_ms[2] the metric FFTs (momentum draw, drift, kinetic energy),
 *   phase_ms[3] everything else (heatbath, noise, kicks, energies). */
#define HMC_MAX_SOLVES 256
typedef struct {
    int n_solves;                       /* force solves in the trajectory (entries past HMC_MAX_SOLVES are not kept) */
    int reliable_updates;               /* FP64 true-residual evaluations over all solves */
    int iterations[HMC_MAX_SOLVES];     /* inner iterations of each solve (slowest right-hand side) */
    double true_resid[HMC_MAX_SOLVES];  /* final FP64 true relative residual of each solve (worst right-hand side) */
    double phase_ms[4];
} hmc_traj_stats;

/* Copies the record of the last trajectory() of `chain` into *out (host). Errors: HMC_ERR_ARG;
 * HMC_ERR_STATE if the chain has not run a trajectory. */
int hmc_trajectory_stats(const hmc_ctx* ctx, int chain, hmc_traj_stats* out);

/* Tracing: *kernel_launches receives the number of kernels this context has launched since
 * hmc_init (host-side count, no synchronisation). */
int hmc_counters(const hmc_ctx* ctx, int64_t* kernel_launches);

/* Measured arithmetic peak of the current device's CUDA cores, in flop/s (an FMA counts two):
 * dependent fused multiply-add chains in FP64 (prec = HMC_FP64) or FP32 (HMC_FP32), 8 chains
 * per thread, 8 blocks of 256 threads per SM, best of four timed launches on a private stream.
 * The roofline denominator of FP64-bound kernels. Allocates and frees a small scratch buffer;
 * not for use inside stream capture. Errors: HMC_ERR_ARG, HMC_ERR_CUDA. */
int hmc_fma_peak(int prec, double* flop_per_s);

/* Launch plan of the complex64 strip kernel of A = D D^dagger (Eq. linsys) for an L x L x Nt
 * lattice (L a multiple of 16 up to 80), nrhs right-hand sides (1..64) and `slots` resident
 * blocks (SMs x blocks per SM; not in the paper). Right-hand side k runs in nch[k] time chunks of
 * the Nt slices, each chunk as L/16 strip blocks; right-hand sides are launched in the order
 * order[0..nrhs-1], and *nblk receives the launch's block count. The chunk counts are the ones
 * whose greedy dealing of blocks to the slots, a block costing its chunk length + 1.5 slice steps,
 * ends first. nch and order (caller-owned, nrhs entries) are overwritten. Host only: no device
 * work, usable without a GPU. Errors: HMC_ERR_ARG. */
int hmc_strip_plan(int L, int Nt, int nrhs, int slots, int* nch, int* order, int* nblk);

/* Index checks of a library built with -DHMC_BOUNDS: the operator, force and strip kernels check
 * their global and shared-memory indices, record a failed check in a device error word and skip
 * the access (no trap). *word receives the OR of the codes recorded since the last call (1: D
 * operator, 2: force, 4: strip kernel global access, 8: strip kernel shared access) and clears
 * them; *enabled (may be NULL) is 1 in the bounds build. In the normal build *word is 0 and the
 * checks compile to nothing. Synchronises the device. */
int hmc_bounds_status(unsigned int* word, int* enabled);

/* Counter-based random numbers used by HMC_NOISE_PHILOX: Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 * philox_raw: out[4j .. 4j+3] (device uint32) = Philox4x32-10(key, ctr + j), the 128-bit
 *   counter ctr[0] (least significant word) .. ctr[3] advanced by j; key word 0 is the
 *   low half of key. For known-answer tests.
 * philox_normal: n standard normals (complex_out = 0: n doubles) or n standard complex
 *   normals (complex_out = 1: n complex128 with parts N(0, 1/2)) into device memory out.
 *   Block j of the stream (seed, counter) is Philox(key = seed, ctr = {lo j, hi j,
 *   lo counter, hi counter}); each block gives two 53-bit uniforms and, by Box-Muller,
 *   two normals. */
int philox_raw(hmc_ctx* ctx, uint64_t key, const uint32_t ctr[4], int64_t nblocks, void* out);
int philox_normal(hmc_ctx* ctx, uint64_t seed, uint64_t counter, int64_t n, int complex_out,
                  void* out);

#ifdef __cplusplus
}
#endif
#endif /* HMC_H */
