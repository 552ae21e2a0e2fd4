"""Chain-rule GBS sampler (Sec. III) served by the C ABI's worker (gbsh_sampler_*).

`pure_state(U, r, alpha)` builds, with torch on the GPU, the quantities the sampler needs
for a pure Gaussian state (squeezed vacuum with squeezing r through interferometer U, then
displaced to mean amplitudes alpha), following Sec. II with hbar = 2:
  covariance V = S S^T (S = interferometer x squeezer, quadratures (q, p)),
  Sigma = F V F^dag, Q = Sigma + I/2, A = conj(X (I - Q^{-1})) = B (+) B*,
  gamma = Q^{-1} alpha_vec (its first half fills the diagonal in Eq. lhaf-pure),
  (A is read as the conjugate of the printed X (I - Q^{-1}): only then do B and gamma form
  the consistent pair whose loop hafnians give the state's Fock amplitudes),
  p(vac) = exp(-alpha_vec^dag Q^{-1} alpha_vec / 2) / sqrt(det Q),
  Husimi covariance V_Q = V + I restricted to modes 2..M and its Cholesky factor
  (Eq. heterodyne), for the heterodyne draw of step 2.
Mixed states (step 1 of Sec. III): `mixed_state(V, R)` splits V = T + W by the Williamson
decomposition (Eq. split) and describes the state as a mixture of pure states with
covariance T and displacement drawn from N(R, W) (Eqs. decomp, mnpdf). The kernel matrix B
and the heterodyne factor come from T; each sample draws its own displacement, whose fill
vector is the linear map gamma(R) = [Q_T^{-1} F]_{1..M} R.
`Sampler` wraps gbsh_sampler_create/submit/poll/wait/destroy.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import lib as _lib


@dataclass
class PureState:
    B: np.ndarray           # M x M kernel matrix of Eq. lhaf-pure
    gamma: np.ndarray       # M fill vector
    p_vac: float
    het_mean: np.ndarray    # 2(M-1) Husimi means of (q_2..q_M, p_2..p_M)
    het_chol: np.ndarray    # 2(M-1) x 2(M-1) lower Cholesky factor of V_Q on modes 2..M


def pure_state(U, r, alpha, device=None) -> PureState:
    import torch
    dev = torch.device(device) if device is not None else (
        torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu"))
    U = torch.as_tensor(np.asarray(U), dtype=torch.complex128, device=dev)
    r = torch.as_tensor(np.asarray(r, dtype=np.float64), device=dev)
    alpha = torch.as_tensor(np.asarray(alpha), dtype=torch.complex128, device=dev)
    M = U.shape[0]
    hbar = 2.0
    # symplectic of the squeezers (q squeezed) followed by the interferometer a -> U a
    Sr = torch.diag(torch.cat([torch.exp(-r), torch.exp(r)]))
    SU = torch.cat([torch.cat([U.real, -U.imag], 1), torch.cat([U.imag, U.real], 1)], 0)
    S = SU @ Sr
    V = (hbar / 2) * S @ S.T
    R = (2 * hbar) ** 0.5 * torch.cat([alpha.real, alpha.imag])
    eye = torch.eye(M, dtype=torch.complex128, device=dev)
    F = torch.cat([torch.cat([eye, 1j * eye], 1), torch.cat([eye, -1j * eye], 1)], 0) / (2 * hbar) ** 0.5
    Sigma = F @ V.to(torch.complex128) @ F.conj().T
    Q = Sigma + torch.eye(2 * M, dtype=torch.complex128, device=dev) / 2
    Qinv = torch.linalg.inv(Q)
    zero = torch.zeros((M, M), dtype=torch.complex128, device=dev)
    X = torch.cat([torch.cat([zero, eye], 1), torch.cat([eye, zero], 1)], 0)
    A = (X @ (torch.eye(2 * M, dtype=torch.complex128, device=dev) - Qinv)).conj()
    avec = F @ R.to(torch.complex128)
    gvec = Qinv @ avec
    pvac = torch.exp(-0.5 * (avec.conj() @ Qinv @ avec)).real / torch.sqrt(torch.linalg.det(Q)).real
    B = A[:M, :M]
    B = 0.5 * (B + B.T)
    if M > 1:
        rest = list(range(1, M))
        q = rest + [i + M for i in rest]
        VQ = (V + (hbar / 2) * torch.eye(2 * M, dtype=torch.float64, device=dev))[q][:, q]
        L = torch.linalg.cholesky(VQ)
        mean = R[q]
    else:
        L = torch.zeros((0, 0), dtype=torch.float64, device=dev)
        mean = torch.zeros(0, dtype=torch.float64, device=dev)
    return PureState(B=B.cpu().numpy(), gamma=gvec[:M].cpu().numpy(), p_vac=float(pvac),
                     het_mean=mean.cpu().numpy(), het_chol=L.cpu().numpy())


@dataclass
class MixedState:
    B: np.ndarray            # M x M kernel matrix of the pure part T
    het_chol: np.ndarray     # 2(M-1) x 2(M-1) Cholesky factor of T + I on modes 2..M
    fill_map: np.ndarray     # M x 2M complex: fill vector = fill_map @ R
    mean: np.ndarray         # 2M quadrature means R-bar
    w_factor: np.ndarray     # 2M x 2M real, W = w_factor w_factor^T
    nu: np.ndarray           # symplectic eigenvalues (hbar = 2: pure <=> all 1)


def williamson(V):
    """Williamson decomposition V = S^T diag(nu, nu) S (S symplectic w.r.t.
    Omega = [[0, I], [-I, 0]], quadratures (q, p)), from the antisymmetric matrix
    K = V^{-1/2} Omega V^{-1/2}: its eigenpairs of i K (+-d_j) give an orthogonal O with
    O^T K O = [[0, D], [-D, 0]]; then S = D^{1/2} O^T V^{1/2} and nu = 1/d.
    Returns (S, nu) as torch tensors."""
    import torch
    V = V.to(torch.float64)
    m = V.shape[0] // 2
    ev, U = torch.linalg.eigh(V)
    Vh = U @ torch.diag(ev.sqrt()) @ U.T
    Vmh = U @ torch.diag(ev.rsqrt()) @ U.T
    eye = torch.eye(m, dtype=torch.float64, device=V.device)
    zero = torch.zeros((m, m), dtype=torch.float64, device=V.device)
    Om = torch.cat([torch.cat([zero, eye], 1), torch.cat([-eye, zero], 1)], 0)
    K = Vmh @ Om @ Vmh
    w, u = torch.linalg.eigh(1j * K.to(torch.complex128))
    d = w[m:].real                       # the m positive eigenvalues (ascending order)
    up = u[:, m:]
    x = (2 ** 0.5) * up.real             # K x = d y,  K y = -d x
    y = (2 ** 0.5) * up.imag
    O = torch.cat([y, x], 1)
    Dh = torch.cat([d, d]).sqrt()
    S = Dh[:, None] * (O.T @ Vh)
    return S, 1.0 / d


def mixed_state(V, R, device=None) -> MixedState:
    """Gaussian state with quadrature covariance V and means R (hbar = 2) as a mixture of
    pure states (Sec. III step 1)."""
    import torch
    dev = torch.device(device) if device is not None else (
        torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu"))
    V = torch.as_tensor(np.asarray(V, dtype=np.float64), device=dev)
    R = torch.as_tensor(np.asarray(R, dtype=np.float64), device=dev)
    M = V.shape[0] // 2
    S, nu = williamson(V)
    T = S.T @ S                                       # (hbar/2) S^T S with hbar = 2
    excess = torch.clamp(torch.cat([nu, nu]) - 1.0, min=0.0)
    Wf = S.T * excess.sqrt()[None, :]                 # W = S^T (N - I) S = Wf Wf^T
    eye = torch.eye(M, dtype=torch.complex128, device=dev)
    F = torch.cat([torch.cat([eye, 1j * eye], 1), torch.cat([eye, -1j * eye], 1)], 0) / 2.0
    Q = F @ T.to(torch.complex128) @ F.conj().T + torch.eye(2 * M, dtype=torch.complex128, device=dev) / 2
    Qinv = torch.linalg.inv(Q)
    zero = torch.zeros((M, M), dtype=torch.complex128, device=dev)
    X = torch.cat([torch.cat([zero, eye], 1), torch.cat([eye, zero], 1)], 0)
    A = (X @ (torch.eye(2 * M, dtype=torch.complex128, device=dev) - Qinv)).conj()
    B = A[:M, :M]
    B = 0.5 * (B + B.T)
    G = (Qinv @ F)[:M, :]
    if M > 1:
        rest = list(range(1, M))
        q = rest + [i + M for i in rest]
        L = torch.linalg.cholesky((T + torch.eye(2 * M, dtype=torch.float64, device=dev))[q][:, q])
    else:
        L = torch.zeros((0, 0), dtype=torch.float64, device=dev)
    return MixedState(B=B.cpu().numpy(), het_chol=L.cpu().numpy(), fill_map=G.cpu().numpy(),
                      mean=R.cpu().numpy(), w_factor=Wf.cpu().numpy(), nu=nu.cpu().numpy())


def lossy_state(U, r, alpha, eta):
    """Squeezed vacuum (r) through U, displaced to alpha, then uniform loss: transmission
    eta on every mode. Returns (V, R) in quadratures, hbar = 2."""
    U = np.asarray(U, dtype=np.complex128)
    r = np.asarray(r, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.complex128)
    M = len(r)
    Sr = np.diag(np.concatenate([np.exp(-r), np.exp(r)]))
    SU = np.block([[U.real, -U.imag], [U.imag, U.real]])
    S = SU @ Sr
    V = eta * (S @ S.T) + (1 - eta) * np.eye(2 * M)
    R = np.sqrt(eta) * 2.0 * np.concatenate([alpha.real, alpha.imag])
    return V, R


class _Cfg(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int),
                ("gamma", ctypes.c_void_p), ("het_mean", ctypes.c_void_p),
                ("het_chol", ctypes.c_void_p), ("cutoff", ctypes.c_int), ("n_cap", ctypes.c_int),
                ("max_active", ctypes.c_int), ("mem_budget", ctypes.c_size_t),
                ("batching", ctypes.c_int), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("threshold", ctypes.c_int), ("mixed", ctypes.c_int), ("mean", ctypes.c_void_p),
                ("w_factor", ctypes.c_void_p), ("fill_map", ctypes.c_void_p),
                ("tick_subsets", ctypes.c_size_t)]


class ReqStats(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("lhafs", ctypes.c_int), ("ticks", ctypes.c_int), ("truncated", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _bind():
    so = _lib.load()
    if getattr(so, "_gbsh_sampler_bound", False):
        return so
    vp, i = ctypes.c_void_p, ctypes.c_int
    so.gbsh_sampler_create.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(vp)]
    so.gbsh_sampler_submit.argtypes = [vp, ctypes.c_uint64, i, ctypes.POINTER(ctypes.c_uint64)]
    so.gbsh_sampler_poll.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(ReqStats)]
    so.gbsh_sampler_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, vp, ctypes.POINTER(ReqStats)]
    so.gbsh_sampler_cancel.argtypes = [vp, ctypes.c_uint64]
    so.gbsh_sampler_destroy.argtypes = [vp]
    so.gbsh_philox4x32.argtypes = [vp, vp, vp]
    for f in ("gbsh_sampler_create", "gbsh_sampler_submit", "gbsh_sampler_poll",
              "gbsh_sampler_wait", "gbsh_sampler_cancel", "gbsh_sampler_destroy",
              "gbsh_philox4x32"):
        getattr(so, f).restype = i
    so._gbsh_sampler_bound = True
    return so


def philox4x32(counter, key):
    """The library's Philox4x32-10 block function (for verification)."""
    so = _bind()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib._check(so.gbsh_philox4x32(c.ctypes.data, k.ctypes.data, out.ctypes.data), "gbsh_philox4x32")
    return out


class Sampler:
    """A served chain-rule sampler for one pure state."""

    def __init__(self, state, cutoff: int = 4, n_cap: int = 36, max_active: int = 256,
                 mem_budget: int = 2 << 30, batching: bool = True,
                 precision: int = _lib.PREC_FP64, device: int = 0, threshold: bool = False,
                 tick_subsets: int = 0):
        """tick_subsets > 0 splits loop hafnians with more pair subsets than that into fixed
        subset ranges evaluated over several ticks (bounded tick time; see gbsh_sampler_cfg)."""
        self.so = _bind()
        self.M = state.B.shape[0]
        M = self.M
        mixed = isinstance(state, MixedState)
        self._B = np.ascontiguousarray(state.B, dtype=np.complex128)
        self._L = np.ascontiguousarray(state.het_chol, dtype=np.float64)
        if mixed:
            self._g = np.zeros(M, dtype=np.complex128)
            self._m = np.zeros(max(2 * (M - 1), 1), dtype=np.float64)
            self._mean = np.ascontiguousarray(state.mean, dtype=np.float64)
            self._wf = np.ascontiguousarray(state.w_factor, dtype=np.float64)
            self._fm = np.ascontiguousarray(state.fill_map, dtype=np.complex128)
        else:
            self._g = np.ascontiguousarray(state.gamma, dtype=np.complex128)
            self._m = np.ascontiguousarray(state.het_mean, dtype=np.float64)
            self._mean = self._wf = self._fm = None
        cfg = _Cfg(M, self._B.ctypes.data, M, self._g.ctypes.data,
                   self._m.ctypes.data if self._m.size else None,
                   self._L.ctypes.data if self._L.size else None, cutoff, n_cap,
                   max_active if batching else 1, mem_budget, 1 if batching else 0, precision,
                   device, 1 if threshold else 0, 1 if mixed else 0,
                   self._mean.ctypes.data if mixed else None,
                   self._wf.ctypes.data if mixed else None,
                   self._fm.ctypes.data if mixed else None, int(tick_subsets))
        h = ctypes.c_void_p()
        _lib._check(self.so.gbsh_sampler_create(ctypes.byref(cfg), ctypes.byref(h)),
                    "gbsh_sampler_create")
        self.h = h

    def submit(self, seed: int, n_samples: int = 1) -> int:
        rid = ctypes.c_uint64()
        _lib._check(self.so.gbsh_sampler_submit(self.h, seed, n_samples, ctypes.byref(rid)),
                    "gbsh_sampler_submit")
        self._n = getattr(self, "_n", {})
        self._n[rid.value] = n_samples
        return rid.value

    def _result(self, rc, rid, buf, st):
        if rc == _lib.GBSH_PENDING:
            return None
        _lib._check(rc, "gbsh_sampler")
        self._n.pop(rid, None)
        return buf.reshape(-1, self.M), st.as_dict()

    def poll(self, rid: int):
        buf = np.zeros(self._n[rid] * self.M, dtype=np.int32)
        st = ReqStats()
        rc = self.so.gbsh_sampler_poll(self.h, rid, buf.ctypes.data, ctypes.byref(st))
        return self._result(rc, rid, buf, st)

    def wait(self, rid: int, timeout: float = 600.0):
        buf = np.zeros(self._n[rid] * self.M, dtype=np.int32)
        st = ReqStats()
        rc = self.so.gbsh_sampler_wait(self.h, rid, float(timeout), buf.ctypes.data,
                                       ctypes.byref(st))
        return self._result(rc, rid, buf, st)

    def cancel(self, rid: int):
        _lib._check(self.so.gbsh_sampler_cancel(self.h, rid), "gbsh_sampler_cancel")
        self._n.pop(rid, None)

    def close(self):
        if getattr(self, "h", None):
            self.so.gbsh_sampler_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
