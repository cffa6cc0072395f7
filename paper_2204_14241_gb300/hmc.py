"""Thin Python binding of libhmc (include/hmc.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module checks tensor shapes,
dtypes and devices, passes raw device pointers and the CUDA stream, and converts the
returned structs. PyTorch supplies device memory and streams. If libhmc.so is missing
or fails to load, every call raises -- there is no fallback.

Tensor layouts (library layout, see include/hmc.h):
  boson field / momenta / sigma-hat: float64 (3, Nt, L, L) indexed [a, tau, y, x]
  fermion vectors: complex128 or complex64 (nrhs, Nt, L, L, 2, 2) indexed [k, tau, y, x, alpha, s]
"""

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# HMC_LIBRARY selects another build of the same library (the -DHMC_BOUNDS variant)
LIB_PATH = os.environ.get("HMC_LIBRARY", os.path.join(HERE, "libhmc.so"))

HMC_OK, HMC_ERR_ARG, HMC_ERR_NOCONV, HMC_ERR_NONFINITE, HMC_ERR_TIMEOUT, HMC_ERR_CUDA, HMC_ERR_STATE = range(7)
FP64, FP32 = 0, 1
SOLVER_FP64, SOLVER_MIXED = 0, 1
NOISE_EXPLICIT, NOISE_PHILOX = 0, 1
METRIC_MOMENTUM, METRIC_VELOCITY, METRIC_KINETIC, METRIC_ACCUM, METRIC_MNORM = range(5)

# every function declared in include/hmc.h
EXPORTS = ("hmc_init", "hmc_destroy", "hmc_last_error", "hmc_counters", "apply_M", "apply_MdagM",
           "apply_MdagM_static", "apply_precond", "green_estimate",
           "cg_solve", "force", "metric_apply", "trajectory", "hmc_trajectory_stats", "philox_raw", "philox_normal",
           "hmc_fma_peak", "hmc_bounds_status", "hmc_strip_plan")


class HmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libhmc error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Nt", ctypes.c_int), ("dtau", ctypes.c_double),
                ("t_h", ctypes.c_double * 2), ("t_v", ctypes.c_double * 2), ("mu", ctypes.c_double * 2),
                ("g", ctypes.c_double), ("r", ctypes.c_double), ("u", ctypes.c_double), ("c", ctypes.c_double),
                ("solver_mode", ctypes.c_int), ("nrhs_max", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("cg_maxit", ctypes.c_int), ("initial_guess", ctypes.c_int), ("autotune", ctypes.c_int),
                ("wait_spin_limit", ctypes.c_int), ("test_wait_timeout", ctypes.c_int), ("batch_chains", ctypes.c_int),
                ("batch_graph", ctypes.c_int)]


class Chain(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("Nt", ctypes.c_int), ("r", ctypes.c_double)]


class CgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "reliable_updates": self.reliable_updates,
                "converged": bool(self.converged), "true_rel_resid": self.true_rel_resid}


class TrajIn(ctypes.Structure):
    _fields_ = [("phi", ctypes.POINTER(ctypes.c_void_p)), ("sigma_hat", ctypes.POINTER(ctypes.c_void_p)),
                ("eps", ctypes.c_double), ("n_leap", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("precond", ctypes.c_int), ("noise", ctypes.c_int),
                ("chi", ctypes.POINTER(ctypes.c_void_p)), ("z", ctypes.POINTER(ctypes.c_void_p)),
                ("u", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.c_uint64), ("counter", ctypes.c_uint64)]


MAX_SOLVES = 256


class TrajStats(ctypes.Structure):
    _fields_ = [("n_solves", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("iterations", ctypes.c_int * MAX_SOLVES), ("true_resid", ctypes.c_double * MAX_SOLVES),
                ("phase_ms", ctypes.c_double * 4)]

    def as_dict(self):
        n = min(self.n_solves, MAX_SOLVES)
        return {"n_solves": self.n_solves, "reliable_updates": self.reliable_updates,
                "iterations": list(self.iterations[:n]), "true_resid": list(self.true_resid[:n]),
                "phase_ms": dict(zip(("solve", "force", "metric", "other"), self.phase_ms))}


class TrajOut(ctypes.Structure):
    _fields_ = [("dH", ctypes.POINTER(ctypes.c_double)), ("accepted", ctypes.POINTER(ctypes.c_int)),
                ("energies", ctypes.POINTER(ctypes.c_double)), ("cg_iterations", ctypes.POINTER(ctypes.c_int)),
                ("max_true_resid", ctypes.POINTER(ctypes.c_double)), ("jump2", ctypes.POINTER(ctypes.c_double))]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int


def lib():
    """Load libhmc.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "hmc_init": [ctypes.POINTER(Params), _I, ctypes.POINTER(Chain), _P, ctypes.POINTER(_P)],
        "hmc_destroy": [_P],
        "hmc_last_error": [_P],
        "hmc_counters": [_P, ctypes.POINTER(ctypes.c_int64)],
        "apply_M": [_P, _I, _I, _P, _P, _P, _I, _I],
        "apply_MdagM": [_P, _I, _I, _P, _P, _P, _I, ctypes.POINTER(ctypes.c_double)],
        "apply_MdagM_static": [ctypes.POINTER(Params), _I, _I, _I, _P, _P, _P, _I, ctypes.POINTER(ctypes.c_double),
                               _P],
        "apply_precond": [_P, _I, _I, _P, _P, _I],
        "cg_solve": [_P, _I, _P, _P, _P, _I, ctypes.c_double, _I, _I, ctypes.POINTER(CgStats)],
        "force": [_P, _I, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_double), _I, _I,
                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(CgStats)],
        "metric_apply": [_P, _I, _I, _P, _P, _P, ctypes.POINTER(ctypes.c_double)],
        "green_estimate": [_P, _I, _P, _P, _I, _P, _I, ctypes.POINTER(CgStats)],
        "trajectory": [_P, ctypes.POINTER(TrajIn), ctypes.POINTER(TrajOut)],
        "hmc_trajectory_stats": [_P, _I, ctypes.POINTER(TrajStats)],
        "philox_raw": [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64, _P],
        "philox_normal": [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, _I, _P],
        "hmc_fma_peak": [_I, ctypes.POINTER(ctypes.c_double)],
        "hmc_bounds_status": [ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int)],
        "hmc_strip_plan": [_I, _I, _I, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "hmc_last_error" else _I
    _lib = L
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def bounds_status():
    """(word, enabled) of the bounds build's index checks (word 0 and enabled False otherwise)."""
    lib_ = lib()
    w, e = ctypes.c_uint(), ctypes.c_int()
    rc = lib_.hmc_bounds_status(ctypes.byref(w), ctypes.byref(e))
    if rc:
        raise HmcError(rc, lib_.hmc_last_error(None).decode())
    return w.value, bool(e.value)


def strip_plan(L, Nt, nrhs, slots):
    """(nch, order, nblk): the complex64 strip operator's launch plan (libhmc's hmc_strip_plan,
    host only)."""
    lib_ = lib()
    nch, order, nblk = (ctypes.c_int * nrhs)(), (ctypes.c_int * nrhs)(), ctypes.c_int()
    rc = lib_.hmc_strip_plan(L, Nt, nrhs, slots, nch, order, ctypes.byref(nblk))
    if rc:
        raise HmcError(rc, lib_.hmc_last_error(None).decode())
    return list(nch), list(order), nblk.value


def fma_peak(prec=FP64, device=None):
    """Measured FMA throughput (flop/s) of the CUDA cores in FP64 (or FP32) on `device`."""
    lib_ = lib()
    v = ctypes.c_double()
    with torch.cuda.device(torch.device(device or "cuda")):
        rc = lib_.hmc_fma_peak(prec, ctypes.byref(v))
    if rc:
        raise HmcError(rc, lib_.hmc_last_error(None).decode())
    return v.value


def apply_MdagM_static(params, L, Nt, phi, x, out, norms=False, stream=None):
    """y = D D^dagger x without allocating device memory (libhmc's apply_MdagM_static): for
    callers that must not allocate after start-up. `params` is a Params (or a Context's
    .params); `out` is caller-allocated like x. Returns out, or (out, norms) when norms is set."""
    lib_ = lib()
    if x.dtype == torch.complex128:
        prec, rdt = FP64, torch.float64
    elif x.dtype == torch.complex64:
        prec, rdt = FP32, torch.float32
    else:
        raise ValueError("fermion vectors must be complex128 or complex64")
    for name, t in (("phi", phi), ("x", x), ("out", out)):
        if t.device.type != "cuda" or t.device != x.device:
            raise ValueError(f"{name} must be a CUDA tensor on {x.device}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if phi.dtype != rdt or tuple(phi.shape) != (3, Nt, L, L):
        raise ValueError(f"phi must be {rdt} of shape (3, {Nt}, {L}, {L}) for {x.dtype} vectors")
    if x.dim() != 6 or tuple(x.shape[1:]) != (Nt, L, L, 2, 2):
        raise ValueError(f"x must have shape (nrhs, {Nt}, {L}, {L}, 2, 2), got {tuple(x.shape)}")
    if out.dtype != x.dtype or tuple(out.shape) != tuple(x.shape):
        raise ValueError("out must have the dtype and shape of x")
    k = x.shape[0]
    nrm = (ctypes.c_double * k)() if norms else None
    with torch.cuda.device(x.device):
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        rc = lib_.apply_MdagM_static(ctypes.byref(params), L, Nt, prec, _ptr(phi), _ptr(x), _ptr(out), k, nrm,
                                     ctypes.c_void_p(st.cuda_stream))
    if rc:
        raise HmcError(rc, lib_.hmc_last_error(None).decode())
    return (out, list(nrm)) if norms else out


class Context:
    """One libhmc context (hmc_init ... hmc_destroy) bound to a CUDA stream."""

    def __init__(self, L, Nt, dtau=0.1, t_h=(1.0, 0.5), t_v=(0.5, 1.0), mu=(-0.5, -0.5), g=1.0, r=0.5,
                 u=1.0, c=3.0, solver="mixed", nrhs_max=1, cg_tol=1e-10, cg_maxit=100000, chains=None,
                 stream=None, device=None, initial_guess=0, autotune=0, wait_spin_limit=0, test_wait_timeout=0,
                 batch_chains=0, batch_graph=None):
        self.lib = lib()
        self.device = torch.device(device or "cuda")
        p = Params()
        p.L, p.Nt, p.dtau = L, Nt, dtau
        p.t_h[:] = list(t_h)
        p.t_v[:] = list(t_v)
        p.mu[:] = list(mu)
        p.g, p.r, p.u, p.c = g, r, u, c
        p.solver_mode = SOLVER_MIXED if solver == "mixed" else SOLVER_FP64
        p.nrhs_max, p.cg_tol, p.cg_maxit = nrhs_max, cg_tol, cg_maxit
        p.initial_guess = int(initial_guess)
        p.autotune = int(autotune)
        p.wait_spin_limit = int(wait_spin_limit)
        p.test_wait_timeout = int(test_wait_timeout)
        p.batch_chains = int(batch_chains)
        # the batched form replays its leapfrog as a CUDA graph unless asked not to
        p.batch_graph = int(bool(batch_chains) if batch_graph is None else batch_graph)
        self.params = p
        if chains is None:
            chains = [(L, Nt, r)]
        self.chains = [tuple(ch) for ch in chains]
        arr = (Chain * len(chains))(*[Chain(a, b, cc) for (a, b, cc) in chains])
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            rc = self.lib.hmc_init(ctypes.byref(p), len(chains), arr, ctypes.c_void_p(self.stream.cuda_stream),
                                   ctypes.byref(h))
        if rc:
            raise HmcError(rc, self.lib.hmc_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise HmcError(rc, self.lib.hmc_last_error(self.h).decode())

    def launches(self):
        """Kernels launched by this context so far (library-side count)."""
        n = ctypes.c_int64()
        self._check(self.lib.hmc_counters(self.h, ctypes.byref(n)))
        return n.value

    # ---- shape helpers ----------------------------------------------------------------
    def dims(self, chain=0):
        L, Nt, _ = self.chains[chain]
        return L, Nt

    def _boson(self, t, chain, dtype=torch.float64):
        L, Nt = self.dims(chain)
        if t.device.type != "cuda" or t.dtype != dtype or tuple(t.shape) != (3, Nt, L, L) or not t.is_contiguous():
            raise ValueError(f"expected contiguous {dtype} CUDA tensor of shape (3, {Nt}, {L}, {L})")

    def _fermion(self, t, chain, dtype):
        L, Nt = self.dims(chain)
        if t.device.type != "cuda" or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"expected contiguous {dtype} CUDA tensor")
        if t.dim() != 6 or tuple(t.shape[1:]) != (Nt, L, L, 2, 2):
            raise ValueError(f"expected shape (nrhs, {Nt}, {L}, {L}, 2, 2), got {tuple(t.shape)}")
        return t.shape[0]

    @staticmethod
    def _prec(x):
        if x.dtype == torch.complex128:
            return FP64, torch.float64
        if x.dtype == torch.complex64:
            return FP32, torch.float32
        raise ValueError("fermion vectors must be complex128 or complex64")

    # ---- entry points -----------------------------------------------------------------
    def apply_M(self, phi, x, dagger=False, chain=0, out=None):
        prec, rdt = self._prec(x)
        k = self._fermion(x, chain, x.dtype)
        self._boson(phi, chain, rdt)
        y = torch.empty_like(x) if out is None else out
        self._check(self.lib.apply_M(self.h, chain, prec, _ptr(phi), _ptr(x), _ptr(y), int(bool(dagger)), k))
        return y

    def apply_MdagM(self, phi, x, chain=0, norms=False, out=None):
        prec, rdt = self._prec(x)
        k = self._fermion(x, chain, x.dtype)
        self._boson(phi, chain, rdt)
        y = torch.empty_like(x) if out is None else out
        nrm = (ctypes.c_double * k)() if norms else None
        self._check(self.lib.apply_MdagM(self.h, chain, prec, _ptr(phi), _ptr(x), _ptr(y), k, nrm))
        return (y, list(nrm)) if norms else y

    def apply_precond(self, x, chain=0, out=None):
        """y = P x (libhmc's apply_precond); out may be x itself."""
        prec, _ = self._prec(x)
        k = self._fermion(x, chain, x.dtype)
        if out is None:
            y = torch.empty_like(x)
        else:
            self._fermion(out, chain, x.dtype)
            if tuple(out.shape) != tuple(x.shape):
                raise ValueError("out must have the shape of x")
            y = out
        self._check(self.lib.apply_precond(self.h, chain, prec, _ptr(x), _ptr(y), k))
        return y

    def cg_solve(self, phi, b, tol=0.0, maxit=0, precond=True, chain=0, out=None, raise_on_noconv=True):
        k = self._fermion(b, chain, torch.complex128)
        self._boson(phi, chain)
        x = torch.empty_like(b) if out is None else out
        st = CgStats()
        rc = self.lib.cg_solve(self.h, chain, _ptr(phi), _ptr(b), _ptr(x), k, tol, maxit, int(bool(precond)),
                               ctypes.byref(st))
        if rc and (raise_on_noconv or rc != HMC_ERR_NOCONV):
            self._check(rc)
        d = st.as_dict()
        d["status"] = rc
        return x, d

    def force(self, phi, phi_pf, include_boson=True, precond=True, chain=0, out=None):
        k = self._fermion(phi_pf, chain, torch.complex128)
        self._boson(phi, chain)
        F = torch.empty_like(phi) if out is None else out
        spf, sb = ctypes.c_double(), ctypes.c_double()
        st = CgStats()
        self._check(self.lib.force(self.h, chain, _ptr(phi), _ptr(phi_pf), k, _ptr(F), ctypes.byref(spf),
                                   int(bool(include_boson)), int(bool(precond)), ctypes.byref(sb), ctypes.byref(st)))
        return F, spf.value, sb.value, st.as_dict()

    def green_estimate(self, phi, probes, precond=True, chain=0):
        """(1/K) sum_k v_k . (F~^* D^-1 F~ v_k) for K = probes.shape[0] +-1 probes (complex128,
        shape (K, Nt, L, L, 2, 2), twisted Fourier basis). Returns (estimate (Nt, L, L, 2, 2), stats)."""
        k = self._fermion(probes, chain, torch.complex128)
        self._boson(phi, chain)
        out = torch.empty(probes.shape[1:], dtype=torch.complex128, device=probes.device)
        st = CgStats()
        self._check(self.lib.green_estimate(self.h, chain, _ptr(phi), _ptr(probes), k, _ptr(out), int(bool(precond)),
                                            ctypes.byref(st)))
        return out, st.as_dict()

    def metric(self, op, sig, inp, out=None, chain=0):
        self._boson(sig, chain)
        self._boson(inp, chain)
        if op in (METRIC_KINETIC, METRIC_MNORM):
            s = ctypes.c_double()
            self._check(self.lib.metric_apply(self.h, chain, op, _ptr(sig), _ptr(inp), None, ctypes.byref(s)))
            return s.value
        if out is None:
            out = torch.zeros_like(inp) if op == METRIC_ACCUM else torch.empty_like(inp)
        self._check(self.lib.metric_apply(self.h, chain, op, _ptr(sig), _ptr(inp), _ptr(out), None))
        return out

    def trajectory(self, phis, sigmas, eps, n_leap, nrhs=1, precond=True, chi=None, z=None, u=None,
                   seed=None, counter=0, check=True):
        """One HMC update of every chain. phis (list of tensors) are updated in place.
        Explicit noise: chi, z (lists of tensors) and u (list of floats); otherwise Philox
        noise from (seed, counter)."""
        nc = len(self.chains)
        assert len(phis) == nc and len(sigmas) == nc
        for c in range(nc):
            self._boson(phis[c], c)
            self._boson(sigmas[c], c)
        P = ctypes.c_void_p * nc
        ti = TrajIn()
        ti.phi = P(*[t.data_ptr() for t in phis])
        ti.sigma_hat = P(*[t.data_ptr() for t in sigmas])
        ti.eps, ti.n_leap, ti.nrhs, ti.precond = eps, n_leap, nrhs, int(bool(precond))
        if chi is not None:
            for c in range(nc):
                if self._fermion(chi[c], c, torch.complex128) != nrhs:
                    raise ValueError("chi must have nrhs right-hand sides")
                self._boson(z[c], c)
            ti.noise = NOISE_EXPLICIT
            ti.chi = P(*[t.data_ptr() for t in chi])
            ti.z = P(*[t.data_ptr() for t in z])
            ti.u = (ctypes.c_double * nc)(*u)
        else:
            ti.noise = NOISE_PHILOX
            ti.seed, ti.counter = int(seed or 0), int(counter)
        dH = (ctypes.c_double * nc)()
        acc = (ctypes.c_int * nc)()
        en = (ctypes.c_double * (6 * nc))()
        its = (ctypes.c_int * nc)()
        res = (ctypes.c_double * nc)()
        j2 = (ctypes.c_double * nc)()
        to = TrajOut(dH, acc, en, its, res, j2)
        rc = self.lib.trajectory(self.h, ctypes.byref(ti), ctypes.byref(to))
        if check:
            self._check(rc)
        return {"status": rc, "dH": list(dH), "accepted": [bool(a) for a in acc],
                "energies": [list(en[6 * c:6 * c + 6]) for c in range(nc)],
                "cg_iterations": list(its), "max_true_resid": list(res), "jump2": list(j2)}

    def trajectory_stats(self, chain=0):
        """Per-solve iterations and residuals and per-phase GPU times of the chain's last trajectory."""
        st = TrajStats()
        rc = self.lib.hmc_trajectory_stats(self.h, chain, ctypes.byref(st))
        if rc:
            raise HmcError(rc, self.lib.hmc_last_error(None).decode())
        return st.as_dict()

    def philox_raw(self, key, ctr, nblocks):
        out = torch.empty(4 * nblocks, dtype=torch.int64, device=self.device)
        buf = torch.empty(4 * nblocks, dtype=torch.int32, device=self.device)
        c = (ctypes.c_uint32 * 4)(*[v & 0xffffffff for v in ctr])
        self._check(self.lib.philox_raw(self.h, key, c, nblocks, _ptr(buf)))
        out.copy_(buf.to(torch.int64) & 0xffffffff)
        return out

    def philox_normal(self, seed, counter, n, complex_out=False):
        out = torch.empty(n, dtype=torch.complex128 if complex_out else torch.float64, device=self.device)
        self._check(self.lib.philox_normal(self.h, seed, counter, n, int(bool(complex_out)), _ptr(out)))
        return out
