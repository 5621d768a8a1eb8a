"""GB300-native two-site DMRG engine (real-space parallel DMRG, Stoudenmire & White).

Thin ctypes binding over ``libpdmrg.so`` whose C ABI is declared in ``include/pdmrg.h``.
This module only marshals arguments: every step of the DMRG hot path runs in the library's
CUDA kernels.  Device buffers are passed as integer device pointers (e.g. ``tensor.data_ptr()``
of a CUDA torch tensor); streams as integer ``cudaStream_t`` handles (0 = default stream).
The library must be built first (``paper_1301_3494_gb300.build.build()``); importing the
binding never falls back to another implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdmrg.so")

FP64, TF32, BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "tf32": TF32, "bf16": BF16}

_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class MpoDesc(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("d", C.c_int), ("qn_local", _ip), ("D", _ip), ("flux", _ip),
                ("W", _dp), ("qn_total", C.c_int)]


class MpsDesc(C.Structure):
    _fields_ = [("n_sectors", _ip), ("sector_q", _ip), ("sector_m", _ip), ("data", _dp),
                ("canonical", C.c_int), ("center", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("mv_gemm_launches", C.c_longlong), ("mv_gemm_ms", C.c_double),
                ("mv_gemm_flops", C.c_double), ("env_gemm_launches", C.c_longlong), ("env_gemm_ms", C.c_double),
                ("env_gemm_flops", C.c_double), ("f64_gemm_launches", C.c_longlong), ("f64_gemm_ms", C.c_double),
                ("f64_gemm_flops", C.c_double), ("f32_gemm_launches", C.c_longlong), ("f32_gemm_ms", C.c_double),
                ("f32_gemm_flops", C.c_double), ("svd_calls", C.c_longlong), ("svd_sweeps", C.c_longlong),
                ("svd_ms", C.c_double), ("svd_block_calls", C.c_longlong), ("svd_fp64_calls", C.c_longlong),
                ("svd_block_ms", C.c_double), ("svd_fp64_ms", C.c_double), ("svd_max_rows", C.c_longlong),
                ("svd_fp64_fallbacks", C.c_longlong), ("svd_block_flops", C.c_double),
                ("svd_rot_hist", C.c_longlong * 48), ("emu_fallbacks", C.c_longlong), ("tune_classes", C.c_longlong),
                ("tune_changed", C.c_longlong), ("svd_bonds", C.c_longlong), ("svd_block_alg_flops", C.c_double),
                ("svd_block_alg_bytes", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["svd_rot_hist"] = list(d["svd_rot_hist"])
        return d


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("kmax", C.c_int), ("stream", C.c_void_p), ("svd_fp64", C.c_int),
                ("fp64_emulation", C.c_int), ("svd_plain_jacobi", C.c_int), ("env_fp64", C.c_int),
                ("accurate_edges", C.c_int)]


class SweepParams(C.Structure):
    _fields_ = [("m_max", C.c_int), ("dav_tol", C.c_double), ("dav_max_iter", C.c_int), ("refine_iters", C.c_int),
                ("serial_regions", C.c_int)]


class SweepStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_trunc_err", C.c_double), ("max_m", C.c_int),
                ("n_matvec", C.c_int), ("n_steps", C.c_int), ("dav_nonconv", C.c_int),
                ("seconds", C.c_double), ("matvec_seconds", C.c_double), ("matvec_flops", C.c_double),
                ("min_fidelity", C.c_double), ("max_fidelity", C.c_double), ("n_refine_matvec", C.c_int),
                ("refine_seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GemmProblem(C.Structure):
    _fields_ = [("M", C.c_int), ("N", C.c_int), ("seg0", C.c_int), ("nseg", C.c_int), ("c_off", C.c_longlong),
                ("sam", C.c_int), ("sak", C.c_int), ("sbn", C.c_int), ("sbk", C.c_int), ("scm", C.c_int),
                ("scn", C.c_int), ("accumulate", C.c_int), ("pad_", C.c_int), ("alpha", C.c_double)]


class GemmSegment(C.Structure):
    _fields_ = [("a_off", C.c_longlong), ("b_off", C.c_longlong), ("K", C.c_int), ("pad_", C.c_int)]


class BondDesc(C.Structure):
    _fields_ = [("d", C.c_int), ("qn_local", _ip),
                ("nl", C.c_int), ("ql", _ip), ("ml", _ip),
                ("nr", C.c_int), ("qr", _ip), ("mr", _ip),
                ("D0", C.c_int), ("D1", C.c_int), ("D2", C.c_int),
                ("f0", _ip), ("f1", _ip), ("f2", _ip),
                ("W1", _dp), ("W2", _dp)]


class DMRGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)} ({status}): {msg}")
        self.status = status


_lib = None


def lib():
    """Load libpdmrg.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1301_3494_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, st = C.c_void_p, C.c_int
        L.dmrg_status_string.restype = C.c_char_p
        L.dmrg_status_string.argtypes = [C.c_int]
        L.dmrg_last_error.restype = C.c_char_p
        L.dmrg_last_error.argtypes = [vp]
        L.dmrg_init_mpo.argtypes = [C.POINTER(vp), C.POINTER(MpoDesc), C.POINTER(Config)]
        L.dmrg_set_mps.argtypes = [vp, C.POINTER(MpsDesc)]
        L.dmrg_setup_regions.argtypes = [vp, C.c_int, C.c_int, C.POINTER(SweepParams)]
        L.dmrg_sweep.argtypes = [vp, C.POINTER(SweepParams), C.POINTER(SweepStats)]
        L.dmrg_advance.argtypes = [vp, C.c_int, C.POINTER(SweepParams), C.POINTER(SweepStats)]
        L.dmrg_profile_enable.argtypes = [C.c_int]
        L.dmrg_profile_enable.restype = None
        L.dmrg_profile_reset.argtypes = []
        L.dmrg_profile_reset.restype = None
        L.dmrg_profile_read.argtypes = [C.POINTER(Profile)]
        L.dmrg_merge.argtypes = [vp, C.c_int, C.POINTER(SweepParams), _dp, _dp]
        L.dmrg_energy.argtypes = [vp, _dp]
        L.dmrg_get_bond.argtypes = [vp, C.c_int, _ip, _ip, C.c_int, _ip]
        L.dmrg_get_lambda.argtypes = [vp, C.c_int, _dp, C.c_int, _ip]
        L.dmrg_get_center.argtypes = [vp, C.c_int, _ip]
        L.dmrg_get_site.argtypes = [vp, C.c_int, _dp, C.c_longlong, C.POINTER(C.c_longlong)]
        L.dmrg_energy_gradient.argtypes = [vp, _dp, _dp]
        L.dmrg_inverse_canonical.argtypes = [vp]
        L.dmrg_icmps_bond.argtypes = [vp, C.c_int, _ip, _ip, C.c_int, _ip]
        L.dmrg_icmps_v.argtypes = [vp, C.c_int, _dp, C.c_int, _ip]
        L.dmrg_icmps_site.argtypes = [vp, C.c_int, _dp, C.c_longlong, C.POINTER(C.c_longlong)]
        L.dmrg_local_expectations.argtypes = [vp, C.c_int, _dp, _dp, C.c_int, _dp, _dp, C.POINTER(C.c_float)]
        L.dmrg_destroy.argtypes = [vp]
        L.dmrg_heff_apply.argtypes = [C.POINTER(BondDesc), C.c_int, vp, vp, vp, vp, _dp, vp]
        L.dmrg_heff_apply_noalloc.argtypes = [C.POINTER(BondDesc), vp, vp, vp, vp, vp]
        L.dmrg_heff_backward.argtypes = [C.POINTER(BondDesc), vp, vp, vp, vp, vp, vp, vp, _dp, _dp, vp]
        L.dmrg_env_left.argtypes = [C.POINTER(BondDesc), C.c_int, vp, vp, vp, vp]
        L.dmrg_env_right.argtypes = [C.POINTER(BondDesc), C.c_int, vp, vp, vp, vp]
        L.dmrg_gemm64.argtypes = [C.POINTER(GemmProblem), C.c_int, C.POINTER(GemmSegment), C.c_int, vp, vp, vp, C.c_int,
                                  _ip, vp]
        L.dmrg_svd_split.argtypes = [C.POINTER(BondDesc), vp, C.c_int, C.c_int, vp, vp, vp, C.c_int, _ip, _ip, _ip,
                                     _dp, vp]
        L.dmrg_svd_split_batch.argtypes = [C.c_int, C.POINTER(BondDesc), C.POINTER(vp), _ip, C.c_int, C.POINTER(vp),
                                           C.POINTER(vp), C.POINTER(vp), C.c_int, _ip, _ip, _ip, _dp, vp]
        for name in ("dmrg_init_mpo", "dmrg_set_mps", "dmrg_setup_regions", "dmrg_sweep", "dmrg_advance",
                     "dmrg_profile_read", "dmrg_merge",
                     "dmrg_energy", "dmrg_get_bond", "dmrg_get_lambda", "dmrg_get_center", "dmrg_get_site",
                     "dmrg_energy_gradient", "dmrg_destroy", "dmrg_inverse_canonical", "dmrg_icmps_bond",
                     "dmrg_icmps_v", "dmrg_icmps_site", "dmrg_local_expectations",
                     "dmrg_heff_apply", "dmrg_heff_apply_noalloc", "dmrg_heff_backward", "dmrg_env_left",
                     "dmrg_env_right",
                     "dmrg_svd_split", "dmrg_svd_split_batch", "dmrg_gemm64"):
            getattr(L, name).restype = st
        _lib = L
    return _lib


def profile_enable(on=True):
    lib().dmrg_profile_enable(int(bool(on)))


def profile_reset():
    lib().dmrg_profile_reset()


def profile_read():
    p = Profile()
    _check(lib().dmrg_profile_read(C.byref(p)))
    return p.as_dict()


def probe(kind, stream=0):
    """Measured throughput in TFLOP/s (dmrg_probe): 0 FP64 FMA, 1 FP32 FMA, 2 tcgen05 bf16 GEMM 8192^3,
    3 tcgen05 tf32 GEMM 8192^3."""
    v = C.c_double(0.0)
    _check(lib().dmrg_probe(int(kind), C.byref(v), C.c_void_p(stream)))
    return v.value


def status_string(s):
    return lib().dmrg_status_string(int(s)).decode()


def _check(status, ctx=None):
    if status != 0:
        msg = lib().dmrg_last_error(ctx).decode()
        raise DMRGError(status, msg)


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(a, t):
    return a.ctypes.data_as(t)


# ------------------------------------------------------------------------------------------
# Operation-level entry points
# ------------------------------------------------------------------------------------------
class Bond:
    """Host description of one two-site bond (keeps the arrays alive for the C struct)."""

    def __init__(self, qn, left, right, W1, f0, f1, W2=None, f2=None):
        self.qn = _i32(qn)
        self.ql, self.ml = _i32(list(left.keys())), _i32(list(left.values()))
        self.qr, self.mr = _i32(list(right.keys())), _i32(list(right.values()))
        self.W1 = _f64(W1)
        self.f0, self.f1 = _i32(f0), _i32(f1)
        self.W2 = _f64(W2) if W2 is not None else _f64(np.zeros(1))
        self.f2 = _i32(f2) if f2 is not None else _i32(np.zeros(1))
        D0, _, _, D1 = self.W1.shape
        D2 = self.W2.shape[3] if W2 is not None else 1
        self.desc = BondDesc(len(self.qn), _ptr(self.qn, _ip), len(self.ql), _ptr(self.ql, _ip), _ptr(self.ml, _ip),
                             len(self.qr), _ptr(self.qr, _ip), _ptr(self.mr, _ip), D0, D1, D2,
                             _ptr(self.f0, _ip), _ptr(self.f1, _ip), _ptr(self.f2, _ip),
                             _ptr(self.W1, _dp), _ptr(self.W2, _dp))


def heff_apply(bond: Bond, prec, L_dev, R_dev, x_dev, y_dev, stream=0):
    """y = H_eff x on device buffers; returns the algorithmic flop count."""
    fl = C.c_double(0.0)
    _check(lib().dmrg_heff_apply(C.byref(bond.desc), int(prec), L_dev, R_dev, x_dev, y_dev, C.byref(fl), stream))
    return fl.value


def heff_apply_noalloc(bond: Bond, L_dev, R_dev, x_dev, y_dev, stream=0):
    """FP64 y = H_eff x without any device allocation (scratch in a fixed in-library array)."""
    _check(lib().dmrg_heff_apply_noalloc(C.byref(bond.desc), L_dev, R_dev, x_dev, y_dev, stream))


def heff_backward(bond: Bond, L_dev, R_dev, x_dev, ybar_dev, xbar_dev, Lbar_dev, Rbar_dev, want_w=True, stream=0):
    """Gradients of Phi for y = H_eff x given ybar = dPhi/dy (FP64): writes xbar, Lbar, Rbar
    (device) and returns (W1bar, W2bar) as dense numpy arrays (or (None, None))."""
    W1b = np.zeros(bond.W1.shape) if want_w else None
    W2b = np.zeros(bond.W2.shape) if want_w else None
    _check(lib().dmrg_heff_backward(C.byref(bond.desc), L_dev, R_dev, x_dev, ybar_dev, xbar_dev, Lbar_dev, Rbar_dev,
                                    _ptr(W1b, _dp) if want_w else None, _ptr(W2b, _dp) if want_w else None, stream))
    return W1b, W2b


def env_left(bond: Bond, prec, Lin_dev, A_dev, Lout_dev, stream=0):
    _check(lib().dmrg_env_left(C.byref(bond.desc), int(prec), Lin_dev, A_dev, Lout_dev, stream))


def env_right(bond: Bond, prec, Rin_dev, B_dev, Rout_dev, stream=0):
    _check(lib().dmrg_env_right(C.byref(bond.desc), int(prec), Rin_dev, B_dev, Rout_dev, stream))


def svd_split(bond: Bond, psi_dev, m_max, accurate, A_dev, lam_dev, B_dev, cap=4096, stream=0):
    """Returns (middle-bond sectors dict, discarded weight).  accurate: False/0 FP64 Jacobi,
    True/1 with the accurate recursion, 2 the FP32 block-Jacobi split of the mixed-precision engine;
    + 4: the Jacobi on the sector matrices themselves (no QR preconditioning)."""
    nm = C.c_int(0)
    qm = np.zeros(cap, np.int32)
    mm = np.zeros(cap, np.int32)
    tr = C.c_double(0.0)
    _check(lib().dmrg_svd_split(C.byref(bond.desc), psi_dev, int(m_max), int(accurate), A_dev, lam_dev, B_dev,
                                cap, C.byref(nm), _ptr(qm, _ip), _ptr(mm, _ip), C.byref(tr), stream))
    return {int(q): int(m) for q, m in zip(qm[: nm.value], mm[: nm.value])}, tr.value


def svd_split_batch(bonds, psi_devs, m_max, mode, A_devs, lam_devs, B_devs, cap=4096, stream=0):
    """Splits of several bonds in one pass (dmrg_svd_split_batch): lists of Bond, device pointers
    and m_max per bond, one mode for all (as svd_split).  Returns [(middle-bond sectors dict,
    discarded weight)] per bond."""
    n = len(bonds)
    if n == 0:
        return []
    descs = (BondDesc * n)(*[b.desc for b in bonds])
    P = C.c_void_p * n
    nm = np.zeros(n, np.int32)
    qm = np.zeros(n * cap, np.int32)
    mm = np.zeros(n * cap, np.int32)
    tr = np.zeros(n, np.float64)
    mx = np.ascontiguousarray(m_max, np.int32)
    _check(lib().dmrg_svd_split_batch(n, descs, P(*psi_devs), _ptr(mx, _ip), int(mode),
                                      P(*A_devs), P(*lam_devs), P(*B_devs), cap, _ptr(nm, _ip), _ptr(qm, _ip),
                                      _ptr(mm, _ip), _ptr(tr, _dp), stream))
    return [({int(q): int(m) for q, m in zip(qm[b * cap: b * cap + nm[b]], mm[b * cap: b * cap + nm[b]])},
             float(tr[b])) for b in range(n)]


def gemm64(problems, segments, A_dev, B_dev, C_dev, mode=0, stream=0):
    """Grouped FP64 GEMM (dmrg_gemm64).  problems: tuples (M, N, seg0, nseg, c_off, sam, sak, sbn,
    sbk, scm, scn, accumulate, alpha); segments: tuples (a_off, b_off, K).  mode 0: FP64 units,
    1: FP64-accurate emulation on the bf16 tensor cores.  Returns (beta, s, accumulators)."""
    P = (GemmProblem * max(1, len(problems)))()
    for i, t in enumerate(problems):
        M, N, seg0, nseg, c_off, sam, sak, sbn, sbk, scm, scn, acc, alpha = t
        P[i] = GemmProblem(M, N, seg0, nseg, c_off, sam, sak, sbn, sbk, scm, scn, acc, 0, alpha)
    S = (GemmSegment * max(1, len(segments)))()
    for i, (a, b, k) in enumerate(segments):
        S[i] = GemmSegment(a, b, k, 0)
    info = np.zeros(3, np.int32)
    _check(lib().dmrg_gemm64(P, len(problems), S, len(segments), C.c_void_p(A_dev), C.c_void_p(B_dev),
                             C.c_void_p(C_dev), int(mode), _ptr(info, _ip), C.c_void_p(stream)))
    return tuple(int(x) for x in info)


# ------------------------------------------------------------------------------------------
# Context-level engine
# ------------------------------------------------------------------------------------------
class Engine:
    """A DMRG state on the GPU: MPO, MPS, environments, optional real-space regions."""

    def __init__(self, W, flux, D, qn, qtot=0, precision="fp64", kmax=8, stream=0, svd_fp64=False,
                 fp64_emulation=False, svd_plain_jacobi=False, env_fp64=False, accurate_edges=False):
        self._keep = [_f64(W), _i32(flux), _i32(D), _i32(qn)]
        W_, f_, D_, q_ = self._keep
        self.L = len(D_) - 1
        self.qn = [int(x) for x in q_]
        self._wshapes = [(int(D_[j]), len(q_), len(q_), int(D_[j + 1])) for j in range(self.L)]
        desc = MpoDesc(self.L, len(q_), _ptr(q_, _ip), _ptr(D_, _ip), _ptr(f_, _ip), _ptr(W_, _dp), int(qtot))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg = Config(prec, int(kmax), C.c_void_p(stream), int(bool(svd_fp64)), int(bool(fp64_emulation)),
                     int(bool(svd_plain_jacobi)), int(bool(env_fp64)), int(accurate_edges))
        h = C.c_void_p()
        _check(lib().dmrg_init_mpo(C.byref(h), C.byref(desc), C.byref(cfg)))
        self._h = h

    @staticmethod
    def params(m_max, dav_tol=1e-10, dav_max_iter=100, refine_iters=2, serial_regions=0):
        return SweepParams(int(m_max), float(dav_tol), int(dav_max_iter), int(refine_iters), int(serial_regions))

    def set_mps(self, bonds, site_data, center=None):
        """bonds: list of L+1 dicts charge -> dim; site_data: concatenated packed site tensors.
        center=None: the engine canonicalises; center=c: the tensors are already mixed-canonical
        around site c."""
        ns = _i32([len(b) for b in bonds])
        sq = _i32([q for b in bonds for q in b.keys()])
        sm = _i32([m for b in bonds for m in b.values()])
        data = _f64(site_data)
        desc = MpsDesc(_ptr(ns, _ip), _ptr(sq, _ip), _ptr(sm, _ip), _ptr(data, _dp),
                       0 if center is None else 1, 0 if center is None else int(center))
        _check(lib().dmrg_set_mps(self._h, C.byref(desc)), self._h)

    def setup_regions(self, n_regions, warmup, m_max, dav_tol=1e-10, dav_max_iter=100, refine_iters=2,
                      serial_regions=0):
        p = self.params(m_max, dav_tol, dav_max_iter, refine_iters, serial_regions)
        _check(lib().dmrg_setup_regions(self._h, int(n_regions), int(warmup), C.byref(p)), self._h)

    def sweep(self, m_max, dav_tol=1e-10, dav_max_iter=100, refine_iters=2, serial_regions=0):
        """One serial sweep, or with regions set up one real-space parallel sweep (Fig. 4).
        serial_regions: 0 one host thread and stream per region, 1 the regions one after another,
        2 lockstep (every region's t-th bond step together, their splits in one grouped launch)."""
        p = self.params(m_max, dav_tol, dav_max_iter, refine_iters, serial_regions)
        s = SweepStats()
        _check(lib().dmrg_sweep(self._h, C.byref(p), C.byref(s)), self._h)
        return s.as_dict()

    def advance(self, n_steps, m_max, dav_tol=1e-10, dav_max_iter=100, refine_iters=2):
        p = self.params(m_max, dav_tol, dav_max_iter, refine_iters)
        s = SweepStats()
        _check(lib().dmrg_advance(self._h, int(n_steps), C.byref(p), C.byref(s)), self._h)
        return s.as_dict()

    def merge(self, k, m_max, dav_tol=1e-10, dav_max_iter=100, refine_iters=2):
        p = self.params(m_max, dav_tol, dav_max_iter, refine_iters)
        f, e = C.c_double(0), C.c_double(0)
        _check(lib().dmrg_merge(self._h, int(k), C.byref(p), C.byref(f), C.byref(e)), self._h)
        return f.value, e.value

    def energy(self):
        e = C.c_double(0)
        _check(lib().dmrg_energy(self._h, C.byref(e)), self._h)
        return e.value

    def bond(self, b):
        q = np.zeros(8192, np.int32)
        m = np.zeros(8192, np.int32)
        n = C.c_int(0)
        _check(lib().dmrg_get_bond(self._h, int(b), _ptr(q, _ip), _ptr(m, _ip), 8192, C.byref(n)), self._h)
        return {int(a): int(b_) for a, b_ in zip(q[: n.value], m[: n.value])}

    def lam(self, b):
        v = np.zeros(65536)
        n = C.c_int(0)
        _check(lib().dmrg_get_lambda(self._h, int(b), _ptr(v, _dp), 65536, C.byref(n)), self._h)
        return v[: n.value].copy()

    def site(self, j):
        n = C.c_longlong(0)
        st = lib().dmrg_get_site(self._h, int(j), None, 0, C.byref(n))
        if st not in (0, 4):
            _check(st, self._h)
        v = np.zeros(max(1, n.value))
        _check(lib().dmrg_get_site(self._h, int(j), _ptr(v, _dp), v.size, C.byref(n)), self._h)
        return v[: n.value].copy()

    def energy_gradient(self):
        """(dE/dW_j for every site j as arrays shaped like the MPO tensors, E)."""
        shapes = self._wshapes
        Wb = np.zeros(sum(int(np.prod(sh)) for sh in shapes))
        e = C.c_double(0.0)
        _check(lib().dmrg_energy_gradient(self._h, _ptr(Wb, _dp), C.byref(e)), self._h)
        out, off = [], 0
        for sh in shapes:
            k = int(np.prod(sh))
            out.append(Wb[off: off + k].reshape(sh))
            off += k
        return out, e.value

    def inverse_canonical(self):
        """Build the inverse canonical copy of the serial state (every site an orthogonality
        centre, V = 1/Lambda on every bond)."""
        _check(lib().dmrg_inverse_canonical(self._h), self._h)

    def icmps_bond(self, b):
        q = np.zeros(8192, np.int32)
        m = np.zeros(8192, np.int32)
        n = C.c_int(0)
        _check(lib().dmrg_icmps_bond(self._h, int(b), _ptr(q, _ip), _ptr(m, _ip), 8192, C.byref(n)), self._h)
        return {int(a): int(b_) for a, b_ in zip(q[: n.value], m[: n.value])}

    def icmps_v(self, b):
        v = np.zeros(65536)
        n = C.c_int(0)
        _check(lib().dmrg_icmps_v(self._h, int(b), _ptr(v, _dp), 65536, C.byref(n)), self._h)
        return v[: n.value].copy()

    def icmps_site(self, j):
        n = C.c_longlong(0)
        st = lib().dmrg_icmps_site(self._h, int(j), None, 0, C.byref(n))
        if st not in (0, 4):
            _check(st, self._h)
        v = np.zeros(max(1, n.value))
        _check(lib().dmrg_icmps_site(self._h, int(j), _ptr(v, _dp), v.size, C.byref(n)), self._h)
        return v[: n.value].copy()

    def local_expectations(self, ops1=(), ops2=()):
        """(<O_j> [len(ops1), L], <O_{j,j+1}> [len(ops2), L-1], device ms) from the inverse
        canonical copy; ops1 are [d, d] matrices, ops2 [d*d, d*d] (row index s1*d + s2)."""
        d = len(self.qn)
        o1 = _f64(np.asarray(ops1, dtype=np.float64).reshape(-1, d, d))
        o2 = _f64(np.asarray(ops2, dtype=np.float64).reshape(-1, d * d, d * d))
        n1, n2 = o1.shape[0], o2.shape[0]
        e1 = np.zeros((max(1, n1), self.L))
        e2 = np.zeros((max(1, n2), max(1, self.L - 1)))
        ms = C.c_float(0.0)
        _check(lib().dmrg_local_expectations(self._h, n1, _ptr(o1, _dp), _ptr(e1, _dp), n2, _ptr(o2, _dp),
                                             _ptr(e2, _dp), C.byref(ms)), self._h)
        return e1[:n1], e2[:n2, : self.L - 1], ms.value

    def state(self):
        """(bonds, packed site data, centre) of the serial state, for set_mps."""
        bonds = [self.bond(b) for b in range(self.L + 1)]
        data = np.concatenate([self.site(j) for j in range(self.L)])
        return bonds, data, self.center()

    def region_state(self):
        """(bonds, packed site data) of the real-space parallel state (every boundary's V in the
        first site to its right); not canonical: load it with set_mps(bonds, data)."""
        bonds = [self.bond(b) for b in range(self.L + 1)]
        data = np.concatenate([self.site(j) for j in range(self.L)])
        return bonds, data

    def center(self, region=0):
        s = C.c_int(0)
        _check(lib().dmrg_get_center(self._h, int(region), C.byref(s)), self._h)
        return s.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dmrg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
