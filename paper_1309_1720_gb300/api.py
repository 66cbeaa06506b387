"""Python binding of the GB300 FP64 cardiac stepper.

Thin wrappers over the C ABI (include/cardiac_gb300.h): problems become
``cg_problem`` records, torch CUDA tensors supply device pointers and
streams, and every step of the computation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import CProblem, CTuning, check

# enums of cardiac_gb300.h
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ENAN, ETIMEOUT, EUNSUPPORTED = range(8)
FHN, BOCF, KARMA, DIFFUSION = 0, 1, 2, 3
STENCIL5, STENCIL9 = 0, 1
MIRROR, CLAMP, PERIODIC = 0, 1, 2
EULER, HEUN, RK4, RUSH_LARSEN, IMPLICIT_EULER = 0, 1, 2, 3, 4
FLAG_ALLOW_UNSTABLE = 1 << 0
FLAG_PER_STAGE_LAUNCH = 1 << 1
FLAG_NEIGHBOR_SYNC = 1 << 2
FLAG_TANH_AS_HK = 1 << 3
FLAG_TEST_STUCK_BARRIER = 1 << 8
DEV_NONFINITE, DEV_TIMEOUT = 1, 2
ABI_VERSION = 1

_DEFAULT_D = {FHN: (1.0, 1.5), BOCF: (1.171e-3,), KARMA: (1.1e-3,), DIFFUSION: (1.0,)}


def n_fields(model: int) -> int:
    return int(_lib.lib().cg_n_fields(model))


def n_params(model: int) -> int:
    return int(_lib.lib().cg_n_params(model))


def default_params(model: int):
    n = n_params(model)
    buf = (ctypes.c_double * max(n, 1))()
    check(_lib.lib().cg_default_params(model, buf))
    return [buf[i] for i in range(n)]


@dataclass
class Problem:
    """One grid instance: the paper's problem statement (model, grid, D, dt,
    scheme).  ``D`` sets Dxx = Dyy per field; ``Dyy`` overrides for an
    anisotropic diagonal tensor."""
    model: int = FHN
    nx: int = 128
    ny: int = 128
    dx: float = 0.04
    dy: Optional[float] = None
    D: Optional[Sequence[float]] = None
    Dyy: Optional[Sequence[float]] = None
    stencil: int = STENCIL5
    bc: int = MIRROR
    scheme: int = EULER
    alpha_d: float = 1.0 / 6.0
    dt: float = 2e-4
    params: Optional[Sequence[float]] = None
    flags: int = 0
    barrier_timeout_s: float = 0.0
    _keep: list = field(default_factory=list, repr=False, compare=False)

    def to_c(self) -> CProblem:
        c = CProblem()
        c.abi_version = ABI_VERSION
        c.model = self.model
        c.nx, c.ny = int(self.nx), int(self.ny)
        c.dx = float(self.dx)
        c.dy = float(self.dx if self.dy is None else self.dy)
        Dxx = list(_DEFAULT_D.get(self.model, ()) if self.D is None else self.D)
        Dyy = list(Dxx if self.Dyy is None else self.Dyy)
        for i in range(4):
            c.Dxx[i] = float(Dxx[i]) if i < len(Dxx) else 0.0
            c.Dyy[i] = float(Dyy[i]) if i < len(Dyy) else 0.0
        c.stencil, c.bc, c.scheme = self.stencil, self.bc, self.scheme
        c.flags = self.flags
        c.alpha_d = float(self.alpha_d)
        c.dt = float(self.dt)
        if self.params is not None:
            arr = (ctypes.c_double * len(self.params))(*[float(x) for x in self.params])
            self._keep = [arr]
            c.params = ctypes.cast(arr, _lib.c_dp)
            c.n_params = len(self.params)
        else:
            c.params = None
            c.n_params = 0
        c.barrier_timeout_s = float(self.barrier_timeout_s)
        return c


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _state(t, numel, name, cuda=True):
    """``t`` if it is a contiguous float64 tensor on the device (host when
    ``cuda`` is False) with ``numel`` elements (any count when None); raises
    TypeError / ValueError otherwise.  The C ABI sees only pointers, so these
    checks keep every kernel inside the buffers it is given."""
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64, got %s" % (name, t.dtype))
    if bool(t.is_cuda) != cuda:
        raise ValueError("%s must be a %s tensor" % (name, "CUDA" if cuda else "CPU"))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return t


class Plan:
    """An immutable stepping plan for one instance or a packed batch.

    The underlying C plan may be shared by calls on several streams, each
    with its own workspace.  This object keeps one device workspace of its
    own that ``run`` (without ``workspace=``), ``rhs``, ``tlm`` and
    ``adjoint`` reuse, so calls that may overlap on different streams either
    pass ``workspace=`` to ``run`` or use separate Plan objects."""

    def __init__(self, problems, tuning: Optional[dict] = None):
        L = _lib.lib()
        single = isinstance(problems, Problem)
        self.problems = [problems] if single else list(problems)
        self.tuning = dict(tuning) if tuning else None
        self.model = self.problems[0].model
        self.nv = n_fields(self.model)
        cprobs = (CProblem * len(self.problems))(*[p.to_c() for p in self.problems])
        tun = None
        if tuning:
            tun = CTuning(int(tuning.get("cells_x", 0)), int(tuning.get("rows", 0)),
                          int(tuning.get("threads", 0)), int(tuning.get("blocks_per_sm", 0)),
                          int(tuning.get("schedule", 0)))
        h = ctypes.c_void_p()
        if single:
            st = L.cg_plan_create_tuned(cprobs, ctypes.byref(tun) if tun else None, ctypes.byref(h))
        else:
            st = L.cg_batch_create(cprobs, len(self.problems), ctypes.byref(tun) if tun else None,
                                   ctypes.byref(h))
        check(st)
        self._h = h
        n = L.cg_plan_n_instances(h)
        offs = (ctypes.c_int64 * (n + 1))()
        check(L.cg_batch_offsets(h, offs))
        self.offsets = [int(offs[i]) for i in range(n + 1)]
        sz = ctypes.c_size_t()
        check(L.cg_workspace_size(h, ctypes.byref(sz)))
        self.workspace_bytes = int(sz.value)
        self._ws = None
        self._host_ws = None

    # -- resources
    @property
    def handle(self):
        return self._h

    def workspace(self) -> torch.Tensor:
        """The plan's own device workspace (zero-filled when allocated, so its
        status word reads 0 before the first run)."""
        if self._ws is None:
            self._ws = torch.zeros(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        return self._ws

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.lib().cg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout helpers
    def shape(self, i: int = 0):
        p = self.problems[i]
        return (self.nv, int(p.ny), int(p.nx))

    def pack(self, states) -> torch.Tensor:
        """Concatenate per-instance [n_v, ny, nx] tensors into the packed layout."""
        return torch.cat([torch.as_tensor(s, dtype=torch.float64).reshape(-1) for s in states]).cuda()

    def unpack(self, packed: torch.Tensor):
        return [packed[self.offsets[i]:self.offsets[i + 1]].view(self.shape(i))
                for i in range(len(self.problems))]

    # -- stepping
    def run(self, z_in: torch.Tensor, n_steps: int, out: Optional[torch.Tensor] = None,
            stream=None, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Advance by n_steps; returns ``out`` (allocated if None)."""
        _state(z_in, self.offsets[-1], "z_in")
        out = torch.empty_like(z_in) if out is None else _state(out, self.offsets[-1], "out")
        if workspace is None:
            ws = self.workspace()
        elif not (isinstance(workspace, torch.Tensor) and workspace.is_cuda and workspace.is_contiguous()
                  and workspace.numel() * workspace.element_size() >= self.workspace_bytes):
            raise ValueError("workspace must be a contiguous CUDA tensor of at least %d bytes"
                             % self.workspace_bytes)
        else:
            ws = workspace
        check(_lib.lib().cg_run(self._h, z_in.data_ptr(), out.data_ptr(), int(n_steps), ws.data_ptr(),
                                _stream_handle(stream)))
        return out

    def rhs(self, z: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """F(z) = D L z + N[z], the right-hand side the steps integrate."""
        _state(z, self.offsets[-1], "z")
        out = torch.empty_like(z) if out is None else _state(out, self.offsets[-1], "out")
        check(_lib.lib().cg_rhs(self._h, z.data_ptr(), out.data_ptr(), self.workspace().data_ptr(),
                                _stream_handle(stream)))
        return out

    def run_batch(self, states, n_steps: int, outs=None, stream=None):
        """Advance each instance in its own device tensor (``states[i]`` of
        shape [n_v, ny, nx]); returns the output tensors (``outs`` or new ones;
        ``outs[i] is states[i]`` steps in place)."""
        n = len(self.problems)
        if len(states) != n:
            raise ValueError("%d states for a plan of %d instances" % (len(states), n))
        for i, z in enumerate(states):
            _state(z, self.offsets[i + 1] - self.offsets[i], "states[%d]" % i)
        outs = [torch.empty_like(z) for z in states] if outs is None else list(outs)
        if len(outs) != n:
            raise ValueError("%d outputs for a plan of %d instances" % (len(outs), n))
        for i, o in enumerate(outs):
            _state(o, self.offsets[i + 1] - self.offsets[i], "outs[%d]" % i)
        pin = (ctypes.c_void_p * n)(*[z.data_ptr() for z in states])
        pout = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        ws = self.workspace()
        check(_lib.lib().cg_batch_run(self._h, pin, pout, int(n_steps), ws.data_ptr(), _stream_handle(stream)))
        return outs

    def run_host(self, z_in: torch.Tensor, n_steps: int, out: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
        """Advance a state held in host memory (a CPU float64 tensor, ideally
        pinned): copy in, step, copy out, wait.  Returns ``out`` (a CPU
        tensor, allocated if None; may be ``z_in``)."""
        _state(z_in, self.offsets[-1], "z_in", cuda=False)
        out = torch.empty_like(z_in) if out is None else _state(out, self.offsets[-1], "out", cuda=False)
        sz = ctypes.c_size_t()
        check(_lib.lib().cg_host_workspace_size(self._h, ctypes.byref(sz)))
        if self._host_ws is None or self._host_ws.numel() < sz.value:
            self._host_ws = torch.zeros(int(sz.value), dtype=torch.uint8, device="cuda")
        check(_lib.lib().cg_run_host(self._h, z_in.data_ptr(), out.data_ptr(), int(n_steps),
                                     self._host_ws.data_ptr(), _stream_handle(stream)))
        return out

    def tlm_workspace(self, n_tangents: int) -> torch.Tensor:
        sz = ctypes.c_size_t()
        check(_lib.lib().cg_tlm_workspace_size(self._h, int(n_tangents), ctypes.byref(sz)))
        if self._ws is None or self._ws.numel() < sz.value:
            self._ws = torch.zeros(max(int(sz.value), self.workspace_bytes), dtype=torch.uint8, device="cuda")
        return self._ws

    def tlm(self, z0: torch.Tensor, dz0: torch.Tensor, n_steps: int, zT: Optional[torch.Tensor] = None,
            dzT: Optional[torch.Tensor] = None, stream=None):
        """Exact Jacobian-vector products of the n-step flow map: returns
        (zT, dzT) with dzT[i] = dPhi/dz(z0) dz0[i]; dz0 is [T, n_v, ny, nx]."""
        N = self.offsets[-1]
        _state(z0, N, "z0")
        _state(dz0, None, "dz0")
        n_t = dz0.numel() // N
        if n_t * N != dz0.numel():
            raise ValueError("dz0 has %d elements, not a multiple of the state's %d" % (dz0.numel(), N))
        zT = torch.empty_like(z0) if zT is None else _state(zT, N, "zT")
        dzT = torch.empty_like(dz0) if dzT is None else _state(dzT, n_t * N, "dzT")
        ws = self.tlm_workspace(n_t)
        check(_lib.lib().cg_tlm_run(self._h, z0.data_ptr(), dz0.data_ptr(), zT.data_ptr(), dzT.data_ptr(),
                                    n_t, int(n_steps), ws.data_ptr(), _stream_handle(stream)))
        return zT, dzT

    def linearize(self, z0: torch.Tensor, n_steps: int, max_tangents: int = 1, stream=None) -> "Linearization":
        """Advance z0 by n_steps keeping every stage's local Jacobian, for
        repeated exact Jacobian-vector products at z0 (``Linearization``)."""
        return Linearization(self, z0, n_steps, max_tangents, stream)

    def adjoint(self, z0: torch.Tensor, lamT: torch.Tensor, n_steps: int, checkpoint_every: int = 0,
                stream=None, with_dD: bool = True):
        """Reverse-mode derivative of the n-step flow map: returns
        (lam0, dLdD) with lam0 = dL/dz0 for lamT = dL/dzT and dLdD the
        derivatives w.r.t. each diffusive field's D (device tensors).
        ``with_dD=False`` skips the dL/dD accumulation (dLdD is None; lam0
        is the same bit for bit)."""
        _state(z0, self.offsets[-1], "z0")
        _state(lamT, self.offsets[-1], "lamT")
        self._adjoint_workspace(n_steps, checkpoint_every)
        lam0 = torch.empty_like(lamT)
        nd = 2 if self.model == FHN else 1
        dLdD = torch.empty(nd, dtype=torch.float64, device="cuda") if with_dD else None
        check(_lib.lib().cg_adjoint_run(self._h, z0.data_ptr(), lamT.data_ptr(), lam0.data_ptr(),
                                        dLdD.data_ptr() if with_dD else None,
                                        int(n_steps), int(checkpoint_every), self._ws.data_ptr(),
                                        _stream_handle(stream)))
        return lam0, dLdD

    def forward_checkpointed(self, z0: torch.Tensor, n_steps: int, checkpoint_every: int = 0, stream=None):
        """z0 -> zT as ``run`` (bit for bit), keeping the checkpoints a later
        gradient needs (cg_adjoint_forward).  Returns (zT, Checkpoints);
        ``Checkpoints.adjoint`` gives what ``adjoint`` would from z0 without
        repeating the forward sweep."""
        _state(z0, self.offsets[-1], "z0")
        ck = Checkpoints(self, int(n_steps), int(checkpoint_every))
        zT = torch.empty_like(z0)
        check(_lib.lib().cg_adjoint_forward(self._h, z0.data_ptr(), zT.data_ptr(), ck.n_steps, ck.every,
                                            ck.buf.data_ptr(), self.workspace().data_ptr(),
                                            _stream_handle(stream)))
        return zT, ck

    def _adjoint_workspace(self, n_steps: int, checkpoint_every: int) -> torch.Tensor:
        sz = ctypes.c_size_t()
        check(_lib.lib().cg_adjoint_workspace_size(self._h, int(n_steps), int(checkpoint_every), ctypes.byref(sz)))
        if self._ws is None or self._ws.numel() < sz.value:
            self._ws = torch.zeros(max(int(sz.value), self.workspace_bytes), dtype=torch.uint8, device="cuda")
        return self._ws

    def newton_step(self, z0: torch.Tensor, period_steps: int, restart: int = 30, max_restarts: int = 1,
                    rtol: float = 1e-10, linearized: bool = False, stream=None):
        """One Newton step on the period-T flow map by GMRES(restart) with
        exact Jacobian-vector products (``linearized``: from stored stage
        Jacobians, no primal work per Krylov iteration; same result).
        Returns (dz, residual_history)."""
        _state(z0, self.offsets[-1], "z0")
        L = _lib.lib()
        sz = ctypes.c_size_t()
        if linearized:
            check(L.cg_newton_linearized_workspace_size(self._h, int(restart), int(period_steps), ctypes.byref(sz)))
        else:
            check(L.cg_newton_workspace_size(self._h, int(restart), ctypes.byref(sz)))
        ws = torch.zeros(int(sz.value), dtype=torch.uint8, device="cuda")
        dz = torch.empty_like(z0)
        hist = (ctypes.c_double * (restart * max_restarts + 1))()
        nit = ctypes.c_int32()
        step = L.cg_newton_gmres_step_linearized if linearized else L.cg_newton_gmres_step
        check(step(self._h, z0.data_ptr(), int(period_steps), int(restart), int(max_restarts), float(rtol),
                   dz.data_ptr(), hist, ctypes.byref(nit), ws.data_ptr(), _stream_handle(stream)))
        return dz, [hist[i] for i in range(nit.value + 1)]

    def status(self, stream=None, workspace: Optional[torch.Tensor] = None, raise_on_error: bool = True) -> int:
        """Device status flags of the last run on ``workspace`` (default: the
        plan's own; 0 if nothing has run on it yet).  Raises CGError on a
        timeout or a non-finite value unless ``raise_on_error`` is False."""
        if workspace is None and self._ws is None:
            return 0
        ws = self.workspace() if workspace is None else workspace
        flags = ctypes.c_uint32()
        st = _lib.lib().cg_read_status(self._h, ws.data_ptr(), _stream_handle(stream), ctypes.byref(flags))
        if raise_on_error:
            check(st)
        return int(flags.value)


class Checkpoints:
    """The checkpoints of one forward run z0 -> zT of a plan
    (``Plan.forward_checkpointed``), in a device buffer of their own;
    ``adjoint`` gives (lam0, dLdD) for a cotangent lamT = dL/dzT, bit for bit
    those of ``Plan.adjoint(z0, lamT, ...)``, with no forward sweep
    (cg_adjoint_reverse).  It only reads the checkpoints, so it may be called
    several times."""

    def __init__(self, plan: Plan, n_steps: int, every: int):
        self.plan = plan
        self.n_steps = n_steps
        self.every = every
        sz = ctypes.c_size_t()
        check(_lib.lib().cg_adjoint_checkpoint_size(plan._h, n_steps, every, ctypes.byref(sz)))
        self.buf = torch.empty(max(int(sz.value) // 8, 1), dtype=torch.float64, device="cuda")

    def adjoint(self, lamT: torch.Tensor, stream=None, with_dD: bool = True):
        p = self.plan
        _state(lamT, p.offsets[-1], "lamT")
        ws = p._adjoint_workspace(self.n_steps, self.every)
        lam0 = torch.empty_like(lamT)
        nd = 2 if p.model == FHN else 1
        dLdD = torch.empty(nd, dtype=torch.float64, device="cuda") if with_dD else None
        check(_lib.lib().cg_adjoint_reverse(p._h, self.buf.data_ptr(), lamT.data_ptr(), lam0.data_ptr(),
                                            dLdD.data_ptr() if with_dD else None, self.n_steps, self.every,
                                            ws.data_ptr(), _stream_handle(stream)))
        return lam0, dLdD


class Linearization:
    """The stage Jacobians of one base trajectory z0 -> zT of a plan
    (cg_tlm_linearize), kept in a workspace of their own; ``apply`` gives
    dPhi/dz(z0) dz0 for up to ``max_tangents`` tangents at a time with no
    primal work (cg_tlm_apply), bit for bit the tangents of ``Plan.tlm``."""

    def __init__(self, plan: Plan, z0: torch.Tensor, n_steps: int, max_tangents: int = 1, stream=None):
        _state(z0, plan.offsets[-1], "z0")
        self.plan = plan
        self.n_steps = int(n_steps)
        self.max_tangents = int(max_tangents)
        sz = ctypes.c_size_t()
        check(_lib.lib().cg_tlm_linearized_workspace_size(plan._h, self.max_tangents, self.n_steps,
                                                          ctypes.byref(sz)))
        self.ws = torch.zeros(int(sz.value), dtype=torch.uint8, device="cuda")
        self.zT = torch.empty_like(z0)
        check(_lib.lib().cg_tlm_linearize(plan._h, z0.data_ptr(), self.zT.data_ptr(), self.n_steps,
                                          self.ws.data_ptr(), _stream_handle(stream)))

    def apply(self, dz0: torch.Tensor, dzT: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """dzT[i] = dPhi/dz(z0) dz0[i]; dz0 is [T, n_v, ny, nx] (or one state)."""
        N = self.zT.numel()
        _state(dz0, None, "dz0")
        n_t = dz0.numel() // N
        if n_t * N != dz0.numel() or n_t > self.max_tangents:
            raise ValueError("dz0 must hold 1..%d states of %d elements, got %d elements"
                             % (self.max_tangents, N, dz0.numel()))
        dzT = torch.empty_like(dz0) if dzT is None else _state(dzT, n_t * N, "dzT")
        check(_lib.lib().cg_tlm_apply(self.plan._h, dz0.data_ptr(), dzT.data_ptr(), n_t, self.n_steps,
                                      self.ws.data_ptr(), _stream_handle(stream)))
        return dzT

    def status(self, stream=None) -> int:
        """Device status of the linearizing and applying runs (raises on error)."""
        return self.plan.status(stream=stream, workspace=self.ws)
