"""Thin ctypes binding of the C ABI in include/tjm.h (argument marshalling only).

Every step of the tensor jump method runs inside libtjm.so on the GPU; this
module converts numpy arrays to the C structures and checks status codes.  It
raises if the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtjm.so")

TJM_OK, TJM_EINVAL, TJM_ENOMEM, TJM_ENUMERIC, TJM_ETIMEOUT, TJM_EBUSY, TJM_EINTERNAL, TJM_ECUDA = range(8)
PREC_FP64, PREC_FP32, PREC_FP32_DEC32, PREC_FP32_DF64 = 0, 1, 2, 3
STATE_ZERO, STATE_PRODUCT, STATE_PRODUCT_PER_TRAJ, STATE_MPS = 0, 1, 2, 3
STATUS_NAMES = {0: "TJM_OK", 1: "TJM_EINVAL", 2: "TJM_ENOMEM", 3: "TJM_ENUMERIC", 4: "TJM_ETIMEOUT",
                5: "TJM_EBUSY", 6: "TJM_EINTERNAL", 7: "TJM_ECUDA"}


class tjm_mpo(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_int), ("D", C.POINTER(C.c_int)), ("W", C.POINTER(C.c_double))]


class tjm_jump(C.Structure):
    _fields_ = [("site", C.c_int), ("rate", C.c_double), ("op", C.c_double * 8)]


class tjm_observable(C.Structure):
    _fields_ = [("site", C.c_int), ("op", C.c_double * 8)]


class tjm_observable2(C.Structure):
    _fields_ = [("site", C.c_int), ("op", C.c_double * 32)]


class tjm_state(C.Structure):
    _fields_ = [("kind", C.c_int), ("data", C.POINTER(C.c_double)), ("chi", C.POINTER(C.c_int))]


class tjm_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("krylov_max", C.c_int), ("krylov_tol", C.c_double),
                ("exact_full_bond", C.c_int), ("device", C.c_int), ("max_ctas", C.c_int),
                ("energy_shift", C.c_int), ("tile_rule", C.c_int), ("tensor_cores", C.c_int),
                ("trotter_order", C.c_int), ("projection_error", C.c_int), ("tc_min_work", C.c_int64)]


class tjm_stats(C.Structure):
    _fields_ = [("n_traj", C.c_int64), ("steps_done_min", C.c_int64), ("steps_done_max", C.c_int64),
                ("failed", C.c_int64), ("matvec_one_site", C.c_uint64), ("matvec_two_site", C.c_uint64),
                ("matvec_bond", C.c_uint64), ("env_updates", C.c_uint64), ("krylov_capped", C.c_uint64),
                ("jumps", C.c_uint64), ("min_margin_jump", C.c_double), ("min_margin_pick", C.c_double),
                ("final_bond_sum", C.c_int64), ("final_bond_max", C.c_int64),
                ("flops_contract", C.c_double), ("flops_decomp", C.c_double), ("cycles", C.c_uint64 * 12)]

    PHASES = ("gemm", "mpo_contract", "lanczos", "qr", "svd", "dissipate_jump", "measure", "tdvp", "env_build",
              "krylov_expm", "matvec", "init")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "cycles"}
        d["cycles"] = {n: int(self.cycles[i]) for i, n in enumerate(self.PHASES)}
        return d


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("tjm_default_options", None, [C.POINTER(tjm_options)]),
    ("tjm_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(tjm_mpo), C.POINTER(tjm_jump), C.c_int, C.c_double,
                             C.c_int, C.c_double, C.POINTER(tjm_options)]),
    ("tjm_run", C.c_int, [C.c_void_p, C.POINTER(tjm_state), C.c_int64, C.c_int64, C.c_uint64,
                          C.POINTER(tjm_observable), C.c_int, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int64)]),
    ("tjm_run_prepare", C.c_int, [C.c_void_p, C.POINTER(tjm_state), C.c_int64, C.c_int64, C.c_uint64,
                                  C.POINTER(tjm_observable), C.c_int, C.POINTER(C.c_double), C.c_int,
                                  C.POINTER(C.c_int64)]),
    ("tjm_run_prepare2", C.c_int, [C.c_void_p, C.POINTER(tjm_state), C.c_int64, C.c_int64, C.c_uint64,
                                   C.POINTER(tjm_observable), C.c_int, C.POINTER(tjm_observable2), C.c_int,
                                   C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int64)]),
    ("tjm_run2", C.c_int, [C.c_void_p, C.POINTER(tjm_state), C.c_int64, C.c_int64, C.c_uint64,
                           C.POINTER(tjm_observable), C.c_int, C.POINTER(tjm_observable2), C.c_int,
                           C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int64)]),
    ("tjm_run_advance", C.c_int, [C.c_void_p, C.c_int64, C.c_int]),
    ("tjm_run_group_advance", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.c_int, C.c_int]),
    ("tjm_poll", C.c_int, [C.c_void_p, C.c_int64]),
    ("tjm_scratch_bytes", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    ("tjm_resident_ctas", C.c_int, [C.c_void_p]),
    ("tjm_result", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.POINTER(C.c_double)]),
    ("tjm_run_stats", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(tjm_stats)]),
    ("tjm_run_margins", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tjm_run_bonds", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int)]),
    ("tjm_run_get_state", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)]),
    ("tjm_run_set_state", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_double)]),
    ("tjm_run_status", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int)]),
    ("tjm_run_set_tile_rule", C.c_int, [C.c_void_p, C.c_int64, C.c_int]),
    ("tjm_wait", C.c_int, [C.c_void_p, C.c_int64, C.c_double]),
    ("tjm_run_free", C.c_int, [C.c_void_p, C.c_int64]),
    ("tjm_stream", C.c_void_p, [C.c_void_p]),
    ("tjm_sync", C.c_int, [C.c_void_p]),
    ("tjm_destroy", None, [C.c_void_p]),
    ("tjm_last_error", C.c_char_p, [C.c_void_p]),
    ("tjm_launch_count", C.c_int64, [C.c_void_p]),
    ("tjm_selftest_qr", C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    ("tjm_selftest_svd", C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tjm_selftest_tc_cgemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tjm_selftest_contract", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("tjm_selftest_expm_tridiag", C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                                            C.POINTER(C.c_double)]),
    ("tjm_selftest_philox", C.c_int, [C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32),
                                      C.POINTER(C.c_uint32), C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libtjm.so (built by paper_2501_17913_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libtjm.so not found at %s: build it with paper_2501_17913_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class TJMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _op8(op):
    op = np.asarray(op, dtype=np.complex128).reshape(2, 2)
    arr = (C.c_double * 8)()
    flat = np.stack([op.real, op.imag], axis=-1).reshape(-1)
    for i in range(8):
        arr[i] = float(flat[i])
    return arr


def _cplx(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1).reshape(-1))


class Context:
    """One TJM problem (tjm_create) and the runs started on it."""

    def __init__(self, W, jumps, dt, chi_max, trunc_eps, precision=PREC_FP32_DF64, krylov_max=30, krylov_tol=0.0,
                 exact=False, device=0, max_ctas=0, energy_shift=True, tile_rule=0, tensor_cores=False,
                 trotter_order=2, projection_error=False, tc_min_work=0):
        lib = load()
        self.lib = lib
        L = len(W)
        D = [1] + [int(np.shape(w)[1]) for w in W]
        self._D = np.array(D, dtype=np.int32)
        self._W = _cplx(np.concatenate([np.asarray(w, dtype=np.complex128).reshape(-1) for w in W]))
        mpo = tjm_mpo(L, 2, self._D.ctypes.data_as(C.POINTER(C.c_int)), _dp(self._W))
        js = (tjm_jump * max(1, len(jumps)))()
        for i, (site, op, rate) in enumerate(jumps):
            js[i].site = int(site)
            js[i].rate = float(rate)
            js[i].op = _op8(op)
        opt = tjm_options()
        lib.tjm_default_options(C.byref(opt))
        opt.precision, opt.krylov_max, opt.krylov_tol = precision, krylov_max, krylov_tol
        opt.exact_full_bond, opt.device, opt.max_ctas = int(bool(exact)), device, max_ctas
        opt.energy_shift = int(bool(energy_shift))
        opt.tile_rule = int(tile_rule)
        opt.tensor_cores = int(bool(tensor_cores))
        opt.trotter_order = int(trotter_order)
        opt.projection_error = int(bool(projection_error))
        opt.tc_min_work = int(tc_min_work)
        self.projection_error = bool(projection_error)
        h = C.c_void_p()
        st = lib.tjm_create(C.byref(h), C.byref(mpo), js, len(jumps), float(dt), int(chi_max), float(trunc_eps),
                            C.byref(opt))
        if st != TJM_OK:
            raise TJMError(st, "tjm_create failed")
        self.h = h
        self.L = L
        self.precision = precision
        self.chi_max = int(chi_max)
        self.runs = {}

    def _check(self, st, what):
        if st != TJM_OK:
            raise TJMError(st, "%s: %s" % (what, self.lib.tjm_last_error(self.h).decode()))

    def _state(self, psi0, n_traj):
        """psi0: None (|0..0>), [L][2] product, [n_traj][L][2] product per trajectory,
        or (chi list, [site tensors]) for an MPS."""
        keep = []
        if psi0 is None:
            return tjm_state(STATE_ZERO, None, None), keep
        if isinstance(psi0, tuple):
            chi, sites = psi0
            chi = np.asarray(chi, dtype=np.int32)
            data = _cplx(np.concatenate([np.asarray(s, dtype=np.complex128).reshape(-1) for s in sites]))
            keep += [chi, data]
            return tjm_state(STATE_MPS, _dp(data), chi.ctypes.data_as(C.POINTER(C.c_int))), keep
        a = np.asarray(psi0, dtype=np.complex128)
        data = _cplx(a)
        keep.append(data)
        kind = STATE_PRODUCT if a.ndim == 2 else STATE_PRODUCT_PER_TRAJ
        if kind == STATE_PRODUCT_PER_TRAJ and a.shape[0] != n_traj:
            raise ValueError("per-trajectory initial states must have n_traj rows")
        return tjm_state(kind, _dp(data), None), keep

    def prepare(self, psi0, n_traj, seed, observables, times, first_traj=0, launch=False):
        """observables: [(site, op)] with op 2 x 2 (one site) or 4 x 4 (sites site, site + 1); results come
        back in the caller's order."""
        st_, keep = self._state(psi0, n_traj)
        one = [(i, s_, o) for i, (s_, o) in enumerate(observables) if np.shape(o) == (2, 2)]
        two = [(i, s_, o) for i, (s_, o) in enumerate(observables) if np.shape(o) == (4, 4)]
        if len(one) + len(two) != len(observables):
            raise ValueError("observables must be 2 x 2 or 4 x 4")
        obs = (tjm_observable * max(1, len(one)))()
        for k, (_, site, op) in enumerate(one):
            obs[k].site = int(site)
            obs[k].op = _op8(op)
        obs2 = (tjm_observable2 * max(1, len(two)))()
        for k, (_, site, op) in enumerate(two):
            obs2[k].site = int(site)
            flat = np.stack([np.asarray(op).real, np.asarray(op).imag], axis=-1).reshape(-1)
            for q in range(32):
                obs2[k].op[q] = float(flat[q])
        t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
        rid = C.c_int64()
        f = self.lib.tjm_run2 if launch else self.lib.tjm_run_prepare2
        st = f(self.h, C.byref(st_), int(n_traj), int(first_traj), C.c_uint64(seed), obs, len(one), obs2, len(two),
               _dp(t), len(t), C.byref(rid))
        self._check(st, "tjm_run" if launch else "tjm_run_prepare")
        # device column of each caller observable: the one-site ones first, then the two-site ones
        order = [i for (i, _, _) in one] + [i for (i, _, _) in two]
        if self.projection_error:
            order.append(len(observables))        # the projection error stays the last column
        inv = np.argsort(order) if order else np.zeros(0, dtype=int)
        self.runs[rid.value] = (int(n_traj), len(t), len(order), inv)
        return rid.value

    def run(self, psi0, n_traj, seed, observables, times, first_traj=0):
        return self.prepare(psi0, n_traj, seed, observables, times, first_traj, launch=True)

    def advance(self, run_id, max_steps):
        self._check(self.lib.tjm_run_advance(self.h, run_id, int(max_steps)), "tjm_run_advance")

    def wait(self, run_id, timeout_s):
        """True once the run's device work has finished, False if it is still running after timeout_s."""
        st = self.lib.tjm_wait(self.h, run_id, float(timeout_s))
        if st == TJM_ETIMEOUT:
            return False
        self._check(st, "tjm_wait")
        return True

    def poll(self, run_id):
        st = self.lib.tjm_poll(self.h, run_id)
        if st == TJM_EBUSY:
            return False
        self._check(st, "tjm_poll")
        return True

    def result(self, run_id, per_traj=True, allow_numeric=False):
        n_traj, n_t, n_o, inv = self.runs[run_id]
        mean = np.zeros((n_t, n_o))
        sem = np.zeros((n_t, n_o))
        pt = np.zeros((n_traj, n_t, n_o)) if per_traj else None
        st = self.lib.tjm_result(self.h, run_id, _dp(mean), _dp(sem), _dp(pt))
        if not (allow_numeric and st == TJM_ENUMERIC):
            self._check(st, "tjm_result")
        if n_o:
            mean, sem = mean[:, inv], sem[:, inv]
            if pt is not None:
                pt = pt[:, :, inv]
        return mean, sem, pt

    def stats(self, run_id):
        s = tjm_stats()
        self._check(self.lib.tjm_run_stats(self.h, run_id, C.byref(s)), "tjm_run_stats")
        return s.as_dict()

    def margins(self, run_id):
        n_traj = self.runs[run_id][0]
        m1 = np.zeros(n_traj)
        m2 = np.zeros(n_traj)
        self._check(self.lib.tjm_run_margins(self.h, run_id, _dp(m1), _dp(m2)), "tjm_run_margins")
        return m1, m2

    def bonds(self, run_id):
        n_traj = self.runs[run_id][0]
        chi = np.zeros((n_traj, self.L + 1), dtype=np.int32)
        self._check(self.lib.tjm_run_bonds(self.h, run_id, chi.ctypes.data_as(C.POINTER(C.c_int))), "tjm_run_bonds")
        return chi

    def get_state(self, run_id, traj):
        """(completed steps, bond dims, [site tensors (chi_l, 2, chi_r)]) of one trajectory."""
        chi = np.zeros(self.L + 1, dtype=np.int32)
        data = np.zeros(2 * self.L * 2 * 64 * 64)
        step = C.c_int()
        self._check(self.lib.tjm_run_get_state(self.h, run_id, int(traj), C.byref(step),
                                               chi.ctypes.data_as(C.POINTER(C.c_int)), _dp(data)), "tjm_run_get_state")
        z = data[0::2] + 1j * data[1::2]
        sites, off = [], 0
        for l in range(self.L):
            n = int(chi[l]) * 2 * int(chi[l + 1])
            sites.append(z[off:off + n].reshape(int(chi[l]), 2, int(chi[l + 1])))
            off += n
        return step.value, chi, sites

    def set_state(self, run_id, traj, step, sites):
        chi = np.array([1] + [int(np.shape(x)[2]) for x in sites], dtype=np.int32)
        data = _cplx(np.concatenate([np.asarray(x, dtype=np.complex128).reshape(-1) for x in sites]))
        self._check(self.lib.tjm_run_set_state(self.h, run_id, int(traj), int(step),
                                               chi.ctypes.data_as(C.POINTER(C.c_int)), _dp(data)), "tjm_run_set_state")

    def status(self, run_id):
        n_traj = self.runs[run_id][0]
        st = np.zeros(n_traj, dtype=np.int32)
        self._check(self.lib.tjm_run_status(self.h, run_id, st.ctypes.data_as(C.POINTER(C.c_int))), "tjm_run_status")
        return st

    def set_tile_rule(self, run_id, rule):
        """GEMM tile rule for the run's later launches (0: 64x64 tiles, 1: 32x32 for small outputs)."""
        self._check(self.lib.tjm_run_set_tile_rule(self.h, run_id, int(rule)), "tjm_run_set_tile_rule")

    def free(self, run_id):
        self._check(self.lib.tjm_run_free(self.h, run_id), "tjm_run_free")
        self.runs.pop(run_id, None)

    def resident_ctas(self):
        """Trajectories in flight in one launch of this context (its kernel's resident wave)."""
        return int(self.lib.tjm_resident_ctas(self.h))

    def scratch_bytes(self, chi_cap, L):
        """Device bytes of the per-CTA scratch a launch holds for trajectories up to (chi_cap, L)."""
        out = C.c_int64()
        self._check(self.lib.tjm_scratch_bytes(self.h, int(chi_cap), int(L), C.byref(out)), "tjm_scratch_bytes")
        return int(out.value)

    def sync(self):
        self._check(self.lib.tjm_sync(self.h), "tjm_sync")

    def stream(self):
        return self.lib.tjm_stream(self.h)

    def launches(self):
        return int(self.lib.tjm_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tjm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def group_advance(pairs, max_steps):
    """One persistent launch over the runs [(Context, run_id), ...]."""
    lib = load()
    n = len(pairs)
    hs = (C.c_void_p * n)(*[p[0].h for p in pairs])
    ids = (C.c_int64 * n)(*[p[1] for p in pairs])
    st = lib.tjm_run_group_advance(hs, ids, n, int(max_steps))
    if st != TJM_OK:
        raise TJMError(st, "tjm_run_group_advance: %s" % lib.tjm_last_error(pairs[0][0].h).decode())


def _z(a):
    return np.ascontiguousarray(a[..., 0] + 1j * a[..., 1])


def selftest_qr(A, double_precision=True):
    """QR of one matrix by the kernel's block routine: returns (Q, R).
    double_precision: False/0 FP32, True/1 FP64, 2 double-float emulated FP64."""
    lib = load()
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    k = min(m, n)
    a = _cplx(A)
    Q = np.zeros((m, k, 2))
    R = np.zeros((k, n, 2))
    st = lib.tjm_selftest_qr(int(double_precision), m, n, _dp(a), _dp(Q), _dp(R))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_qr")
    return _z(Q), _z(R)


def selftest_svd(A, double_precision=True):
    """SVD of one matrix by the kernel's block routine: returns (U, S, V) with A = U diag(S) V^H.
    double_precision: False/0 FP32, True/1 FP64, 2 double-float emulated FP64."""
    lib = load()
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    nn = min(m, n)
    a = _cplx(A)
    U = np.zeros((m, nn, 2))
    V = np.zeros((n, nn, 2))
    S = np.zeros(nn)
    st = lib.tjm_selftest_svd(int(double_precision), m, n, _dp(a), _dp(U), _dp(S), _dp(V))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_svd")
    return _z(U), S, _z(V)


def selftest_tc_cgemm(A, B, conj_a=False, conj_b=False, a_col_major=False, b_k_contig=False):
    """op(A) op(B) by the tensor-core complex GEMM (3xTF32, FP32 accumulation) on one CTA."""
    lib = load()
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    M, K = A.shape
    N = B.shape[1]
    out = np.zeros((M, N, 2))
    st = lib.tjm_selftest_tc_cgemm(M, N, K, int(conj_a), int(conj_b), int(a_col_major), int(b_k_contig),
                                   _dp(_cplx(A)), _dp(_cplx(B)), _dp(out))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_tc_cgemm")
    return _z(out)


def selftest_contract(kind, precision, Lenv, Renv, x, W1=None, W2=None, tensor_cores=True):
    """One effective-Hamiltonian application (kind 0 bond, 1 one site, 2 two sites) or environment update
    (3 left, 4 right) by the trajectory kernel's device functions; layouts as in tjm_selftest_contract."""
    lib = load()
    Lenv = np.asarray(Lenv, dtype=np.complex128)
    Renv = np.asarray(Renv, dtype=np.complex128)
    x = np.asarray(x, dtype=np.complex128)
    if kind == 4:
        chl, chr_ = x.shape[0], x.shape[-1]
        Dl, Dr = np.shape(W1)[0], np.shape(W1)[1]
        Du = 1
    else:
        chl = Lenv.shape[0]
        Dl = Lenv.shape[1]
        chr_ = Renv.shape[2] if kind != 3 else x.shape[-1]
        Dr = Renv.shape[0] if kind in (1, 2) else (np.shape(W1)[1] if kind == 3 else Dl)
        Du = np.shape(W1)[1] if kind == 2 else 1
    shape = {0: (chl, chr_), 1: (chl, 2, chr_), 2: (chl, 2, 2, chr_), 3: (chr_, Dr, chr_), 4: (Dl, chl, chl)}[kind]
    out = np.zeros(shape + (2,))
    w1 = _cplx(W1) if W1 is not None else None
    w2 = _cplx(W2) if W2 is not None else None
    rin = _cplx(Renv) if kind != 3 else np.zeros(2)
    lin = _cplx(Lenv) if kind != 4 else np.zeros(2)
    st = lib.tjm_selftest_contract(int(kind), int(precision), int(bool(tensor_cores)), int(chl), int(chr_), int(Dl),
                                   int(Du), int(Dr), _dp(w1), _dp(w2), _dp(lin), _dp(rin), _dp(_cplx(x)), _dp(out))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_contract")
    return _z(out)


def selftest_expm_tridiag(alpha, beta, theta):
    lib = load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta if len(beta) else [0.0], dtype=np.float64)
    c = np.zeros((len(a), 2))
    st = lib.tjm_selftest_expm_tridiag(len(a), _dp(a), _dp(b), float(theta), _dp(c))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_expm_tridiag")
    return _z(c)


def selftest_philox(seed, traj, step, branch):
    lib = load()
    t = np.ascontiguousarray(traj, dtype=np.uint64)
    s = np.ascontiguousarray(step, dtype=np.uint32)
    b = np.ascontiguousarray(branch, dtype=np.uint32)
    n = len(t)
    u1 = np.zeros(n)
    u2 = np.zeros(n)
    st = lib.tjm_selftest_philox(C.c_uint64(seed), t.ctypes.data_as(C.POINTER(C.c_uint64)),
                                 s.ctypes.data_as(C.POINTER(C.c_uint32)), b.ctypes.data_as(C.POINTER(C.c_uint32)), n,
                                 _dp(u1), _dp(u2))
    if st != TJM_OK:
        raise TJMError(st, "tjm_selftest_philox")
    return u1, u2
