"""GB300-native emRKC solver for the P1 monodomain model (Python binding).

Thin wrapper over the C ABI in include/emrkc.h: it marshals numpy arrays and
CUDA stream handles; every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or no CUDA
device is usable, the calls raise.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _ffi
from ._ffi import Matrix, Options, OwnedMatrix, Stats, Stimulus, Tissue

MODEL_NONE, MODEL_PASSIVE, MODEL_HH, MODEL_TTP06 = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
RHO_ONCE, RHO_FIXED = 0, -1
METHOD_EMRKC, METHOD_EXEX_RL, METHOD_IMEX_RL, METHOD_MRKC = 0, 1, 2, 3


class EmrkcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ffi.ERRORS.get(code, code)}: {msg}")
        self.code = code


def build(verbose=False, force=False):
    from ._buildlib import build as _b
    return _b(verbose=verbose, force=force)


def lib():
    return _ffi.load()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_vars(model: int) -> int:
    return lib().emrkc_num_vars(model)


def num_gates(model: int) -> int:
    return lib().emrkc_num_gates(model)


def rkc_stages(dt, rho, eps=0.05):
    """Algorithm 1 stage count s and interval length beta s^2 (host routine)."""
    s, ls = C.c_int(), C.c_double()
    rc = lib().emrkc_rkc_stages(dt, rho, eps, C.byref(s), C.byref(ls))
    if rc != 0:
        raise EmrkcError(rc, "rkc_stages: invalid arguments")
    return s.value, ls.value


def rkc_coeffs(s, eps=0.05):
    """Algorithm 1 coefficients mu, nu, kappa, c of the s-stage method (host routine)."""
    if s < 1:
        raise EmrkcError(1, "rkc_coeffs: s must be >= 1")
    arrs = [np.zeros(s + 1) for _ in range(4)]
    rc = lib().emrkc_rkc_coeffs(s, eps, *[_dp(a) for a in arrs])
    if rc != 0:
        raise EmrkcError(rc, "rkc_coeffs: invalid arguments")
    return tuple(arrs)


def assemble_p1(coords, cells, D):
    """P1 stiffness K (CSR arrays) and lumped mass by the library's host assembler."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    n, dim = coords.shape
    out = OwnedMatrix()
    rc = lib().emrkc_assemble_p1(dim, n, _dp(coords), cells.shape[0],
                                 cells.ctypes.data_as(C.POINTER(C.c_int64)), _dp(D), C.byref(out))
    if rc != 0:
        raise EmrkcError(rc, "assembly failed")
    try:
        rp = np.ctypeslib.as_array(out.row_ptr, shape=(out.n + 1,)).copy()
        col = np.ctypeslib.as_array(out.col, shape=(max(out.nnz, 1),))[:out.nnz].copy()
        K = np.ctypeslib.as_array(out.K, shape=(max(out.nnz, 1),))[:out.nnz].copy()
        M = np.ctypeslib.as_array(out.lumped_mass, shape=(out.n,)).copy()
    finally:
        lib().emrkc_free_matrix(C.byref(out))
    return rp, col, K, M


def default_options() -> Options:
    o = Options()
    lib().emrkc_default_options(C.byref(o))
    return o


class Solver:
    """One monodomain problem advanced by emRKC on the GPU."""

    def __init__(self, row_ptr, col, K, M, *, chi=1400.0, Cm=1.0, model=MODEL_HH, mask=None,
                 amplitude=50.0, t_on=0.0, t_off=1.0, precision=PREC_FP64, rho_every=1,
                 rho_F=0.0, rho_S=0.0, seed=0, act_threshold=-20.0, stream=None, device=0,
                 profile=False, use_graphs=True, pow_tol=1e-2, pow_max_iter=50, safety=1.05,
                 rho_S_min=0.0, method=0, lin_rtol=1e-10, lin_max_iter=1000, pow_tol_cold=1e-4,
                 pow_max_iter_cold=1000):
        self._lib = lib()
        self._h = C.c_void_p()
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.K = np.ascontiguousarray(K, dtype=np.float64)
        self.M = np.ascontiguousarray(M, dtype=np.float64)
        self.n = self.M.size
        self.model = model
        self.N = num_vars(model)
        mat = Matrix(self.n, self.K.size, self.row_ptr.ctypes.data_as(C.POINTER(C.c_int64)),
                     self.col.ctypes.data_as(C.POINTER(C.c_int32)), _dp(self.K), _dp(self.M))
        tis = Tissue(chi, Cm)
        stim = Stimulus()
        if mask is not None:
            self._mask = np.ascontiguousarray(mask, dtype=np.uint8)
            stim.node_mask = self._mask.ctypes.data_as(C.POINTER(C.c_uint8))
        stim.amplitude = amplitude
        stim.t_on = t_on
        stim.t_off = t_off
        o = default_options()
        o.precision = precision
        o.rho_every = rho_every
        o.rho_F = rho_F
        o.rho_S = rho_S
        o.seed = seed
        o.act_threshold = act_threshold
        o.cuda_stream = stream
        o.device = device
        o.profile = int(profile)
        o.use_graphs = int(use_graphs)
        o.pow_tol = pow_tol
        o.pow_max_iter = pow_max_iter
        o.pow_tol_cold = pow_tol_cold
        o.pow_max_iter_cold = pow_max_iter_cold
        o.safety = safety
        o.rho_S_min = rho_S_min
        o.method = method
        o.lin_rtol = lin_rtol
        o.lin_max_iter = lin_max_iter
        rc = self._lib.emrkc_create(C.byref(mat), C.byref(tis), model, C.byref(stim), C.byref(o),
                                    C.byref(self._h))
        if rc != 0:
            raise EmrkcError(rc, self._lib.emrkc_last_error(None).decode())

    @classmethod
    def from_workload(cls, w, **kw):
        rp, col, K, M = assemble_p1(w.coords, w.cells, w.D)
        return cls(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                   amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off,
                   rho_every=kw.pop("rho_every", w.rho_every), **kw)

    def _check(self, rc):
        if rc != 0:
            raise EmrkcError(rc, self._lib.emrkc_last_error(self._h).decode())

    def step(self, dt):
        self._check(self._lib.emrkc_step(self._h, dt))

    def run(self, T, dt):
        self._check(self._lib.emrkc_run(self._h, T, dt))

    def sync(self):
        self._check(self._lib.emrkc_sync(self._h))
        self._pending = {}

    def get_state(self, var=-1, out=None):
        shape = (self.N, self.n) if var == -1 else (self.n,)
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        self._check(self._lib.emrkc_get_state(self._h, var, _dp(out), out.size))
        return out

    def set_state(self, values, var=-1):
        values = np.ascontiguousarray(values, dtype=np.float64)
        self._check(self._lib.emrkc_set_state(self._h, var, _dp(values), values.size))

    def get_state_device(self, ptr, var, length):
        self._check(self._lib.emrkc_get_state_device(self._h, var, C.c_void_p(ptr), length))

    def set_state_device(self, ptr, var, length):
        self._check(self._lib.emrkc_set_state_device(self._h, var, C.c_void_p(ptr), length))

    def activation_times(self):
        out = np.empty(self.n)
        self._check(self._lib.emrkc_get_activation_times(self._h, _dp(out), self.n))
        return out

    def estimate_rho(self):
        rf, rs = C.c_double(), C.c_double()
        itf, its = C.c_int(), C.c_int()
        self._check(self._lib.emrkc_estimate_rho(self._h, C.byref(rf), C.byref(rs), C.byref(itf),
                                                 C.byref(its)))
        return rf.value, rs.value, itf.value, its.value

    def estimate_rho_F_noalloc(self, d_v, d_w, n, rho_warm=0.0):
        """Algorithm 5 on f_F with caller-owned device vectors (pointers) and the
        library's static scratch; allocates no device memory."""
        rho = C.c_double()
        it = C.c_int()
        self._check(self._lib.emrkc_estimate_rho_F_noalloc(self._h, C.c_void_p(d_v), C.c_void_p(d_w), n,
                                                           rho_warm, C.byref(rho), C.byref(it)))
        return rho.value, it.value

    def set_time(self, t, steps):
        self._check(self._lib.emrkc_set_time(self._h, t, steps))

    def set_stimulus(self, mask, amplitude=50.0, t_on=0.0, t_off=1.0):
        """Replace the applied stimulus (mask of n bytes or None) for the following steps."""
        if mask is None:
            ptr = None
        else:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            ptr = m.ctypes.data_as(C.POINTER(C.c_uint8))
        self._check(self._lib.emrkc_set_stimulus(self._h, ptr, self.n, amplitude, t_on, t_off))

    def set_stimulus_async(self, mask, amplitude=50.0, t_on=0.0, t_off=1.0):
        """set_stimulus without waiting: mask (a C-contiguous uint8 array of n
        bytes, pinned for a truly asynchronous copy) is read by a copy engine
        after the call returns and is kept referenced here until sync()."""
        if mask is None:
            return self.set_stimulus(None, amplitude, t_on, t_off)
        if not (isinstance(mask, np.ndarray) and mask.dtype == np.uint8 and mask.flags.c_contiguous
                and mask.size == self.n):
            raise ValueError("mask must be a C-contiguous uint8 array of n bytes")
        self._check(self._lib.emrkc_set_stimulus_async(self._h, mask.ctypes.data_as(C.POINTER(C.c_uint8)), self.n,
                                                       amplitude, t_on, t_off))
        self._keep(mask)

    def get_state_async(self, var, out):
        """Variable var of the current state into out (a C-contiguous float64
        array of n entries, pinned for a truly asynchronous copy); out is
        complete after sync() and is kept referenced here until then."""
        if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
                and out.size == self.n):
            raise ValueError("out must be a C-contiguous float64 array of n entries")
        self._check(self._lib.emrkc_get_state_async(self._h, var, _dp(out), out.size))
        self._keep(out)
        return out

    def _keep(self, arr):
        # buffers of asynchronous copies stay referenced until the next sync()
        if not hasattr(self, "_pending"):
            self._pending = {}
        self._pending[id(arr)] = arr

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.emrkc_get_stats(self._h, C.byref(st)))
        d = {k: getattr(st, k) for k, _ in Stats._fields_ if k not in ("phase_ms", "phase_launches")}
        d["phase_ms"] = dict(zip(_ffi.PHASES, list(st.phase_ms)))
        d["phase_launches"] = dict(zip(_ffi.PHASES, list(st.phase_launches)))
        return d

    def close(self):
        if self._h:
            self._lib.emrkc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def instance_bytes(n, nnz_per_row, model):
    """Device bytes one batched (mixed-precision) instance holds."""
    return int(lib().emrkc_instance_bytes(int(n), float(nnz_per_row), int(model)))


class Batch:
    """Many monodomain instances advanced together by one persistent launch per step."""

    def __init__(self, *, rho_every=RHO_ONCE, rho_F=0.0, rho_S=0.0, seed=0, act_threshold=-20.0,
                 stream=None, device=0, use_graphs=True):
        self._lib = lib()
        self._h = C.c_void_p()
        o = default_options()
        o.precision = PREC_MIXED
        o.rho_every = rho_every
        o.rho_F = rho_F
        o.rho_S = rho_S
        o.seed = seed
        o.act_threshold = act_threshold
        o.cuda_stream = stream
        o.device = device
        o.use_graphs = int(use_graphs)
        self._rho_every, self._rho_F, self._rho_S = rho_every, rho_F, rho_S
        rc = self._lib.emrkc_batch_create(C.byref(o), C.byref(self._h))
        if rc != 0:
            raise EmrkcError(rc, self._lib.emrkc_batch_last_error(None).decode())
        self._n = {}
        self._N = {}

    def _check(self, rc):
        if rc != 0:
            raise EmrkcError(rc, self._lib.emrkc_batch_last_error(self._h).decode())

    def add(self, row_ptr, col, K, M, *, chi=1400.0, Cm=1.0, model=MODEL_TTP06, mask=None, amplitude=50.0,
            t_on=0.0, t_off=1.0, rho_every=None, rho_F=0.0, rho_S=0.0, rho_S_min=0.0, seed=0,
            act_threshold=-20.0):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        K = np.ascontiguousarray(K, dtype=np.float64)
        M = np.ascontiguousarray(M, dtype=np.float64)
        n = M.size
        mat = Matrix(n, K.size, row_ptr.ctypes.data_as(C.POINTER(C.c_int64)),
                     col.ctypes.data_as(C.POINTER(C.c_int32)), _dp(K), _dp(M))
        tis = Tissue(chi, Cm)
        stim = Stimulus()
        if mask is not None:
            mk = np.ascontiguousarray(mask, dtype=np.uint8)
            stim.node_mask = mk.ctypes.data_as(C.POINTER(C.c_uint8))
        stim.amplitude = amplitude
        stim.t_on = t_on
        stim.t_off = t_off
        o = default_options()
        o.rho_every = self._rho_every if rho_every is None else rho_every
        o.rho_F = rho_F if rho_every is not None else self._rho_F
        o.rho_S = rho_S if rho_every is not None else self._rho_S
        o.rho_S_min = rho_S_min
        o.seed = seed
        o.act_threshold = act_threshold
        out = C.c_int()
        self._check(self._lib.emrkc_batch_add(self._h, C.byref(mat), C.byref(tis), model, C.byref(stim),
                                              C.byref(o), C.byref(out)))
        self._n[out.value] = n
        self._N[out.value] = num_vars(model)
        return out.value

    def add_workload(self, w, **kw):
        rp, col, K, M = assemble_p1(w.coords, w.cells, w.D)
        return self.add(rp, col, K, M, chi=w.chi, Cm=w.Cm, model=w.model, mask=w.stim_mask,
                        amplitude=w.stim_amp, t_on=w.t_on, t_off=w.t_off, **kw)

    def remove(self, iid):
        self._check(self._lib.emrkc_batch_remove(self._h, iid))
        self._n.pop(iid, None)
        self._N.pop(iid, None)

    def step(self, dt):
        self._check(self._lib.emrkc_batch_step(self._h, dt))

    def sync(self):
        self._check(self._lib.emrkc_batch_sync(self._h))

    def get_state(self, iid, var=-1, out=None):
        n, N = self._n[iid], self._N[iid]
        shape = (N, n) if var == -1 else (n,)
        if out is None:
            out = np.empty(shape)
        self._check(self._lib.emrkc_batch_get_state(self._h, iid, var, _dp(out), out.size))
        return out

    def set_state(self, iid, values, var=-1):
        values = np.ascontiguousarray(values, dtype=np.float64)
        self._check(self._lib.emrkc_batch_set_state(self._h, iid, var, _dp(values), values.size))

    def activation_times(self, iid):
        out = np.empty(self._n[iid])
        self._check(self._lib.emrkc_batch_get_activation_times(self._h, iid, _dp(out), out.size))
        return out

    def info(self, iid):
        from ._ffi import BatchInfo
        st = BatchInfo()
        self._check(self._lib.emrkc_batch_get_info(self._h, iid, C.byref(st)))
        return {k: getattr(st, k) for k, _ in BatchInfo._fields_}

    def stats(self):
        from ._ffi import BatchStats
        st = BatchStats()
        self._check(self._lib.emrkc_batch_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in BatchStats._fields_}

    def set_config(self, tile, block):
        self._check(self._lib.emrkc_batch_set_config(self._h, tile, block))

    def set_schedule(self, schedule):
        self._check(self._lib.emrkc_batch_set_schedule(self._h, schedule))

    def set_occupancy(self, threads_per_sm):
        self._check(self._lib.emrkc_batch_set_occupancy(self._h, threads_per_sm))

    def set_spin_limit(self, limit):
        self._check(self._lib.emrkc_batch_set_spin_limit(self._h, limit))

    def autotune(self, dt, reps=3):
        t, b, ms = C.c_int(), C.c_int(), C.c_double()
        self._check(self._lib.emrkc_batch_autotune(self._h, dt, reps, C.byref(t), C.byref(b), C.byref(ms)))
        return t.value, b.value, ms.value

    def ids(self):
        """Instance ids in batch order (the order of the concatenated I/O arrays)."""
        cnt = self._lib.emrkc_batch_ids(self._h, None, 0)
        buf = (C.c_int * max(cnt, 1))()
        self._lib.emrkc_batch_ids(self._h, buf, cnt)
        return list(buf[:cnt])

    def total_nodes(self):
        return int(sum(self._n.values()))

    def set_stimulus_async(self, masks):
        """Node masks of every instance, concatenated in batch order (uint8)."""
        if masks.dtype != np.uint8 or not masks.flags.c_contiguous:
            raise ValueError("masks must be a C-contiguous uint8 array")
        self._check(self._lib.emrkc_batch_set_stimulus_async(
            self._h, masks.ctypes.data_as(C.POINTER(C.c_uint8)), masks.size))

    def get_V_async(self, out):
        """V of every instance, concatenated in batch order, into ``out``
        (float64, complete after sync)."""
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array")
        self._check(self._lib.emrkc_batch_get_V_async(self._h, _dp(out), out.size))

    def get_V32_async(self, out):
        """V of every instance rounded to FP32, concatenated in batch order,
        into ``out`` (float32, complete after sync)."""
        if out.dtype != np.float32 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float32 array")
        self._check(self._lib.emrkc_batch_get_V32_async(self._h, out.ctypes.data_as(C.POINTER(C.c_float)),
                                                        out.size))

    def set_profile(self, on=True):
        self._check(self._lib.emrkc_batch_set_profile(self._h, int(on)))

    def kernel_time(self):
        """(summed ms, launches) of the persistent kernel while profiling."""
        ms, n = C.c_double(), C.c_int64()
        self._check(self._lib.emrkc_batch_get_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def close(self):
        if self._h:
            self._lib.emrkc_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
