"""Thin ctypes binding of the C ABI in include/asd.h (argument marshalling only).

Every computation runs in libasd.so.  Importing this module loads the library and
raises ImportError if it has not been built (``python -m paper_2308_07487_gb300.build``
or ``__graft_entry__.build()``): there is no fallback path.  With ASD_CHECKED=1 in the
environment it loads the index-checked build libasd_checked.so instead
(``build.build(check_bounds=True)``).
Device pointers are passed as integers (e.g. ``tensor.data_ptr()``); streams as
``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_CHECKED = os.environ.get("ASD_CHECKED", "0") == "1"
_SO = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib",
                   "libasd_checked.so" if _CHECKED else "libasd.so")
if not os.path.exists(_SO):
    raise ImportError(f"{os.path.basename(_SO)} not built ({_SO}); run "
                      "paper_2308_07487_gb300/build.py" + (" --checked" if _CHECKED else ""))
lib = ctypes.CDLL(_SO)

ASD_OK, ASD_EINVAL, ASD_ENOMEM, ASD_ECUDA, ASD_ETIMEOUT, ASD_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
ASD_EBOUNDS = -6
ASD_BUILD_CHECK_BOUNDS = 1
ASD_FP32, ASD_TF32, ASD_BF16, ASD_SPLIT_BF16 = 0, 1, 2, 3
PRECISIONS = {"fp32": ASD_FP32, "tf32": ASD_TF32, "bf16": ASD_BF16, "split_bf16": ASD_SPLIT_BF16}
ASD_GEOM_LATTICE, ASD_GEOM_POSITIONS = 0, 1
ASD_METROPOLIS, ASD_HEATBATH, ASD_LEARNED = 0, 1, 2

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_f32p = ctypes.POINTER(ctypes.c_float)
c_f64p = ctypes.POINTER(ctypes.c_double)
c_i64p = ctypes.POINTER(ctypes.c_int64)


class asd_corr_desc(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("n_frames", ctypes.c_int32),
                ("n_samples", ctypes.c_int32), ("T0", ctypes.c_int32), ("n_t", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("center", ctypes.c_int32),
                ("geometry", ctypes.c_int32), ("L", ctypes.c_int32 * 3),
                ("periodic", ctypes.c_int32), ("coords", c_i32p), ("pos", c_f32p),
                ("bin_width", ctypes.c_double), ("n_bins", ctypes.c_int32),
                ("n_q", ctypes.c_int32), ("q", c_f64p), ("tile_n", ctypes.c_int32),
                ("raster_m", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("k_chunks", ctypes.c_int32), ("epi_warps", ctypes.c_int32),
                ("phase_sine", ctypes.c_int32), ("static_schedule", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("cta_pair", ctypes.c_int32)]


class asd_system(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("z", ctypes.c_int32), ("nbr", ctypes.c_void_p),
                ("J", ctypes.c_void_p), ("Hz", ctypes.c_float), ("n_colors", ctypes.c_int32),
                ("color_sites", ctypes.c_void_p), ("color_offsets", c_i64p),
                ("D", ctypes.c_void_p), ("A", ctypes.c_float)]


class asd_mlp(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("W1", ctypes.c_void_p), ("W2", ctypes.c_void_p), ("W3", ctypes.c_void_p),
                ("b1", ctypes.c_void_p), ("b2", ctypes.c_void_p), ("b3", ctypes.c_void_p),
                ("depth", ctypes.c_int32), ("Wm", ctypes.c_void_p), ("bm", ctypes.c_void_p)]


class asd_mc_stats(ctypes.Structure):
    _fields_ = [("proposed", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("cone", ctypes.c_float)]


_VP = ctypes.c_void_p
_SIGS = {
    "asd_pair_corr_plan_create": (ctypes.c_int, [ctypes.POINTER(asd_corr_desc), ctypes.POINTER(_VP)]),
    "asd_pair_corr_plan_destroy": (None, [_VP]),
    "asd_pair_corr_workspace_bytes": (ctypes.c_int64, [_VP]),
    "asd_pair_corr_counts": (ctypes.c_int, [_VP, c_i64p]),
    "asd_pair_corr": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP]),
    "asd_pair_corr_prepare": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.c_int64, _VP]),
    "asd_pair_corr_contract": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP]),
    "asd_pair_corr_contract_range": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64,
                                                    ctypes.c_int32, ctypes.c_int32, _VP, _VP,
                                                    _VP]),
    "asd_pair_corr_batched": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                                             ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    "asd_pair_corr_normalize": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "asd_sync_status": (ctypes.c_int, [_VP]),
    "asd_pair_corr_sq_separable": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "asd_sq_omega": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_double, _VP, ctypes.c_int, _VP, _VP]),
    "asd_selftest_timeout": (ctypes.c_int, [ctypes.c_int64, _VP]),
    "asd_selftest_bounds": (ctypes.c_int, [_VP]),
    "asd_build_flags": (ctypes.c_int, []),
    "asd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "asd_ll_integrate": (ctypes.c_int, [ctypes.POINTER(asd_system), ctypes.c_int, _VP, ctypes.c_float,
                                        ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "asd_ll_integrate_noalloc": (ctypes.c_int, [ctypes.POINTER(asd_system), ctypes.c_int, _VP,
                                                ctypes.c_float, ctypes.c_int, ctypes.c_int, _VP,
                                                _VP, _VP]),
    "asd_thermalize": (ctypes.c_int, [ctypes.POINTER(asd_system), ctypes.c_int, _VP, ctypes.c_float,
                                      ctypes.c_int, ctypes.c_int, ctypes.POINTER(asd_mlp),
                                      ctypes.c_float, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint64, _VP, ctypes.POINTER(asd_mc_stats), _VP]),
    "asd_mlp_param_count": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int]),
    "asd_mlp_param_count_bf16": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int]),
    "asd_mlp_init": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _VP, _VP]),
    "asd_mlp_weights_bf16": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    "asd_mlp_gather": (ctypes.c_int, [ctypes.POINTER(asd_system), ctypes.c_int, _VP, _VP, _VP, _VP]),
    "asd_mlp_loss_grad": (ctypes.c_int, [ctypes.POINTER(asd_mlp), ctypes.c_int64, _VP, _VP, _VP, _VP,
                                         _VP]),
    "asd_mlp_adam_step": (ctypes.c_int, [_VP, _VP, ctypes.c_float, _VP, _VP, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_int, _VP, _VP]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name, None)
    if _f is None:
        continue
    _f.restype = _res
    _f.argtypes = _args


class AsdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {lib.asd_strerror(status).decode()} (status {status})")


def check(status, where="asd"):
    if status != ASD_OK:
        raise AsdError(status, where)
    return status


def strerror(status: int) -> str:
    return lib.asd_strerror(status).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class CorrPlan:
    """Owns an asd_corr_plan.  Geometry arrays are host numpy arrays."""

    def __init__(self, N, F, T0, n_t, precision="split_bf16", S=1, center=False, coords=None,
                 L=(1, 1, 1), periodic=False, pos=None, bin_width=1.0, n_bins=0, q=None,
                 tile_n=0, raster_m=0, stages=0, k_chunks=0, epi_warps=0,
                 phase_sine=False, static_schedule=False, deterministic=False, cta_pair=False):
        d = asd_corr_desc()
        d.n_sites, d.n_frames, d.n_samples, d.T0, d.n_t = N, F, S, T0, n_t
        d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d.center = int(bool(center))
        self._keep = []
        if coords is not None and pos is None:
            d.geometry = ASD_GEOM_LATTICE
            c = np.ascontiguousarray(coords, np.int32)
            self._keep.append(c)
            d.coords = c.ctypes.data_as(c_i32p)
        else:
            d.geometry = ASD_GEOM_POSITIONS
            p = np.ascontiguousarray(pos, np.float32)
            self._keep.append(p)
            d.pos = p.ctypes.data_as(c_f32p)
        for a in range(3):
            d.L[a] = int(L[a])
        d.periodic = int(bool(periodic))
        d.bin_width = float(bin_width)
        d.n_bins = int(n_bins)
        if q is not None and len(q) > 0:
            qq = np.ascontiguousarray(q, np.float64)
            self._keep.append(qq)
            d.n_q = qq.shape[0]
            d.q = qq.ctypes.data_as(c_f64p)
        d.tile_n = int(tile_n)
        d.raster_m = int(raster_m)
        d.stages = int(stages)
        d.k_chunks = int(k_chunks)
        d.epi_warps = int(epi_warps)
        d.phase_sine = int(bool(phase_sine))
        d.static_schedule = int(bool(static_schedule))
        d.deterministic = int(bool(deterministic))
        d.cta_pair = int(bool(cta_pair))
        self.q_parts = 1 + d.phase_sine  # Sq_sum is [n_t][n_q] or [n_t][n_q][2]
        self.desc = d
        self.N, self.F, self.S, self.T0, self.n_t = N, F, S, T0, n_t
        self.n_bins, self.n_q = int(n_bins), int(d.n_q)
        h = _VP()
        check(lib.asd_pair_corr_plan_create(ctypes.byref(d), ctypes.byref(h)), "plan_create")
        self.handle = h
        self._keep = []

    @classmethod
    def for_lattice(cls, lat, F, T0, n_t, w, n_bins, precision="split_bf16", S=1, center=False,
                    q=None, positions=None, **tune):
        """Plan for a synth.Lattice: integer-lattice geometry unless its positions are
        jittered (then the FP32 position rule) or positions=True is forced."""
        jittered = not np.array_equal(lat.pos, lat.coords.astype(np.float32))
        if positions or (positions is None and jittered):
            return cls(lat.n_sites, F, T0, n_t, precision, S, center, pos=lat.pos,
                       bin_width=w, n_bins=n_bins, q=q, **tune)
        return cls(lat.n_sites, F, T0, n_t, precision, S, center, coords=lat.coords, L=lat.L,
                   periodic=lat.periodic, bin_width=w, n_bins=n_bins, q=q, **tune)

    def counts(self):
        out = np.zeros(max(self.n_bins, 1), np.int64)
        check(lib.asd_pair_corr_counts(self.handle, out.ctypes.data_as(c_i64p)), "counts")
        return out[: self.n_bins]

    def workspace_bytes(self):
        return int(lib.asd_pair_corr_workspace_bytes(self.handle))

    def run(self, traj, C_sum=None, Sq_sum=None, rows=None, stream=None):
        r0, r1 = (0, self.N) if rows is None else rows
        check(lib.asd_pair_corr(self.handle, _ptr(traj), r0, r1, _ptr(C_sum), _ptr(Sq_sum),
                                _stream(stream)), "pair_corr")

    def prepare(self, traj, rows=None, stream=None):
        r0, r1 = (0, self.N) if rows is None else rows
        check(lib.asd_pair_corr_prepare(self.handle, _ptr(traj), r0, r1, _stream(stream)),
              "pair_corr_prepare")

    def contract(self, C_sum=None, Sq_sum=None, rows=None, stream=None, t_range=None):
        """asd_pair_corr_contract, or asd_pair_corr_contract_range for the displacements
        t_range = (t_begin, t_end)."""
        r0, r1 = (0, self.N) if rows is None else rows
        if t_range is None:
            check(lib.asd_pair_corr_contract(self.handle, r0, r1, _ptr(C_sum), _ptr(Sq_sum),
                                             _stream(stream)), "pair_corr_contract")
        else:
            check(lib.asd_pair_corr_contract_range(self.handle, r0, r1, int(t_range[0]),
                                                   int(t_range[1]), _ptr(C_sum), _ptr(Sq_sum),
                                                   _stream(stream)), "pair_corr_contract_range")

    def sq_separable(self, traj, Sq_sum, stream=None):
        """asd_pair_corr_sq_separable: the phase-weighted sum through per-site transforms."""
        check(lib.asd_pair_corr_sq_separable(self.handle, _ptr(traj), _ptr(Sq_sum),
                                             _stream(stream)), "pair_corr_sq_separable")

    def normalize(self, C_sum=None, Sq_sum=None, C=None, Sq=None, stream=None):
        check(lib.asd_pair_corr_normalize(self.handle, _ptr(C_sum), _ptr(Sq_sum), _ptr(C), _ptr(Sq),
                                          _stream(stream)), "normalize")

    def close(self):
        if getattr(self, "handle", None):
            lib.asd_pair_corr_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pair_corr_batched(plans, trajs, C_sums, Sq_sums=None, stream=None):
    """asd_pair_corr_batched: every plan's problem in one persistent launch, accumulating
    into C_sums[k] / Sq_sums[k] (device FP64; an entry may be None when its plan has no
    bins / q-vectors, a whole list None when no plan has any).  Preparation is enqueued
    on the same stream.  The work list lives in plans[0]: a CUDA graph captured from a
    repeated call stays valid until plans[0] leads another batch or is closed."""
    n = len(plans)
    P = (_VP * n)(*[p.handle.value for p in plans])
    T = (_VP * n)(*[_ptr(t) for t in trajs])
    C = (_VP * n)(*[_ptr(c) for c in C_sums]) if C_sums is not None else None
    Q = (_VP * n)(*[_ptr(q) for q in Sq_sums]) if Sq_sums is not None else None
    check(lib.asd_pair_corr_batched(P, T, n, C, Q, _stream(stream)), "pair_corr_batched")


WINDOWS = {"none": 0, "hann": 1, "gauss": 2}


def sq_omega(S, dt, omega, Sqw, window="hann", width=0.25, stream=None):
    """asd_sq_omega: S(q, omega) [n_w][n_q] from S(q, t) [n_t][n_q] (device FP64 tensors)."""
    n_t, n_q = S.shape
    check(lib.asd_sq_omega(_ptr(S), int(n_t), int(n_q), float(dt), WINDOWS[window], float(width),
                           _ptr(omega), int(omega.shape[0]), _ptr(Sqw), _stream(stream)),
          "sq_omega")


def sync_status(stream=None):
    return lib.asd_sync_status(_stream(stream))


def selftest_timeout(limit_ns, stream=None):
    """asd_selftest_timeout: a bounded wait that runs out; read with sync_status."""
    check(lib.asd_selftest_timeout(int(limit_ns), _stream(stream)), "selftest_timeout")


def build_flags():
    """asd_build_flags: ASD_BUILD_CHECK_BOUNDS in the index-checked build."""
    return int(lib.asd_build_flags())


def selftest_bounds(stream=None):
    """asd_selftest_bounds (checked build): an index check that fails; read with
    sync_status (ASD_EBOUNDS)."""
    check(lib.asd_selftest_bounds(_stream(stream)), "selftest_bounds")


class Mlp:
    """Learned-proposal network: FP32 master parameters, BF16 weight copy, Adam moments
    (device tensors) and the asd_mlp view the sampler reads.  `depth` = hidden layers of
    64 units (2 or 3).  Without `params` the library draws Glorot-uniform weights from
    `seed` (asd_mlp_init)."""

    def __init__(self, n_in, params=None, device="cuda", seed=0, depth=2):
        import torch
        self.n_in, self.depth = n_in, depth
        P = lib.asd_mlp_param_count(n_in, depth)
        Pw = lib.asd_mlp_param_count_bf16(n_in, depth)
        if P <= 0:
            raise ValueError(f"bad network shape (n_in {n_in}, depth {depth})")
        self.P = P
        self.grad = torch.zeros(P, dtype=torch.float32, device=device)
        self.m = torch.zeros(P, dtype=torch.float32, device=device)
        self.v = torch.zeros(P, dtype=torch.float32, device=device)
        self.wb = torch.zeros(Pw, dtype=torch.bfloat16, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.step = 0
        if params is None:
            self.params = torch.empty(P, dtype=torch.float32, device=device)
            check(lib.asd_mlp_init(_ptr(self.params), n_in, depth, int(seed), _ptr(self.wb),
                                   None), "mlp_init")
        else:
            p = np.asarray(params, np.float32)
            assert p.shape == (P,)
            self.params = torch.from_numpy(p.copy()).to(device)
            self._refresh_bf16()
        # views into the packed vectors: [W1 b1][W2 b2]([Wm bm])[W3 b3] and [W1][W2]([Wm])[W3]
        H, es = 64, self.params.element_size()
        c = asd_mlp()
        c.n_in, c.n_hidden, c.depth = n_in, H, depth
        wp, bs = self.wb.data_ptr(), self.wb.element_size()
        pp = self.params.data_ptr()
        c.W1, c.b1 = wp, pp + H * n_in * es
        c.W2, c.b2 = wp + H * n_in * bs, pp + (H * n_in + H + H * H) * es
        hidden = H * n_in + H + H * H + H          # parameters before the next layer
        wnext = H * n_in + H * H                   # BF16 weights before the next layer
        if depth == 3:
            c.Wm, c.bm = wp + wnext * bs, pp + (hidden + H * H) * es
            hidden += H * H + H
            wnext += H * H
        c.W3, c.b3 = wp + wnext * bs, pp + (hidden + 4 * H) * es
        self.c = c

    def _refresh_bf16(self):
        check(lib.asd_mlp_weights_bf16(_ptr(self.params), self.n_in, self.depth, _ptr(self.wb),
                                       None), "mlp_weights_bf16")

    def loss_grad(self, x, y, n=None, stream=None):
        n = x.shape[0] if n is None else n
        check(lib.asd_mlp_loss_grad(ctypes.byref(self.c), n, _ptr(x), _ptr(y), _ptr(self.grad),
                                    _ptr(self.loss), _stream(stream)), "mlp_loss_grad")

    def adam(self, lr=1e-3, scale=1.0, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.step += 1
        check(lib.asd_mlp_adam_step(_ptr(self.params), _ptr(self.grad), float(scale), _ptr(self.m),
                                    _ptr(self.v), self.n_in, self.depth, float(lr), float(b1),
                                    float(b2), float(eps), self.step, _ptr(self.wb),
                                    _stream(stream)), "mlp_adam_step")


class System:
    """asd_system for a synth.Lattice: neighbour table, couplings and colouring are
    copied to the device (torch tensors kept alive by this object)."""

    def __init__(self, lat, device="cuda"):
        import torch
        self.lat = lat
        self.nbr = torch.from_numpy(np.ascontiguousarray(lat.nbr, np.int32)).to(device)
        self.J = torch.from_numpy(np.ascontiguousarray(lat.J, np.float32)).to(device)
        cs = np.concatenate(lat.colors).astype(np.int32)
        self.color_sites = torch.from_numpy(cs).to(device)
        self.offsets = np.cumsum([0] + [len(c) for c in lat.colors]).astype(np.int64)
        s = asd_system()
        s.n_sites = lat.n_sites
        s.z = lat.nbr.shape[1]
        s.nbr = self.nbr.data_ptr()
        s.J = self.J.data_ptr()
        s.Hz = float(lat.Hz)
        s.n_colors = len(lat.colors)
        s.color_sites = self.color_sites.data_ptr()
        s.color_offsets = self.offsets.ctypes.data_as(c_i64p)
        # Eq. 1's DM vectors per directed bond and single-ion anisotropy (optional)
        D = getattr(lat, "D", None)
        self.D = None if D is None else torch.from_numpy(
            np.ascontiguousarray(D, np.float32)).to(device)
        s.D = self.D.data_ptr() if self.D is not None else None
        s.A = float(getattr(lat, "A", 0.0))
        self.c = s

    def gather(self, spins, x, y, stream=None):
        S = spins.shape[0] if spins.dim() == 3 else 1
        check(lib.asd_mlp_gather(ctypes.byref(self.c), S, _ptr(spins), _ptr(x), _ptr(y),
                                 _stream(stream)), "mlp_gather")

    def ll_integrate(self, spins0, dt, n_frames, stride, traj, spins_out=None, stream=None):
        S = spins0.shape[0] if spins0.dim() == 3 else 1
        check(lib.asd_ll_integrate(ctypes.byref(self.c), S, _ptr(spins0), float(dt), int(n_frames),
                                   int(stride), _ptr(traj), _ptr(spins_out), _stream(stream)),
              "ll_integrate")

    def ll_integrate_noalloc(self, spins0, dt, n_frames, stride, traj, spins_out=None,
                             stream=None):
        """asd_ll_integrate_noalloc: same result, work buffers in the library's fixed
        device array (for callers that cannot allocate; n_sites * n_samples <= 262144)."""
        S = spins0.shape[0] if spins0.dim() == 3 else 1
        check(lib.asd_ll_integrate_noalloc(ctypes.byref(self.c), S, _ptr(spins0), float(dt),
                                           int(n_frames), int(stride), _ptr(traj),
                                           _ptr(spins_out), _stream(stream)),
              "ll_integrate_noalloc")

    def thermalize(self, spins, T, n_sweeps, proposal=ASD_METROPOLIS, net=None, cone=0.0,
                   adapt=False, seed=0, counter=0, uniforms=None, stats=False, stream=None):
        S = spins.shape[0] if spins.dim() == 3 else 1
        st = asd_mc_stats() if stats else None
        check(lib.asd_thermalize(ctypes.byref(self.c), S, _ptr(spins), float(T), int(n_sweeps),
                                 int(proposal), ctypes.byref(net.c) if net is not None else None,
                                 float(cone), int(bool(adapt)), int(seed), int(counter),
                                 _ptr(uniforms), ctypes.byref(st) if st is not None else None,
                                 _stream(stream)), "thermalize")
        return (st.proposed, st.accepted, st.cone) if st is not None else None


def exported_symbols():
    return list(_SIGS)
