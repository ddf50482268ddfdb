"""User-facing wrapper of the librbe2d context: torch tensors in, torch tensors out.

Thin by design: it allocates output tensors with torch and calls the C ABI; every
step of the method runs in librbe2d's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import binding as B


class RBE2D:
    """One random-batch Ewald k-space force context (include/rbe2d.h).

    Geometry and parameters follow the paper's problem statement: cell Lx x Ly, slab
    height H, dielectric contrasts gamma_top / gamma_bot, image levels M, extended
    period Lz, Ewald alpha, real-space cutoff r_c and batch size P.  Negative values
    select the automatic rules (Eq. 3.10 for M, Eq. 3.23 for Lz, (N/(Lx Ly H))^(1/3)
    for alpha, 3/alpha for r_c)."""

    def __init__(self, Lx, Ly, H, *, n_max, P, gamma_top=0.0, gamma_bot=0.0, M=-1, Lz=-1.0, alpha=-1.0,
                 r_c=-1.0, seed=0, eps=1e-4, precision="fp32", coulomb_k=1.0, real_space=False, device=None,
                 stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("RBE2D needs a CUDA device; there is no CPU path")
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.type != "cuda":
            raise ValueError(f"RBE2D runs on a CUDA device, not {dev}")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        prec = {"fp32": B.RBE2D_FP32_MIXED, "fp64": B.RBE2D_FP64}[precision]
        self.precision = precision
        self.out_dtype = torch.float32 if precision == "fp32" else torch.float64
        p = B.rbe2d_params(Lx=Lx, Ly=Ly, H=H, Lz=Lz, gamma_top=gamma_top, gamma_bot=gamma_bot, M=M,
                           alpha=alpha, r_c=r_c, P=P, seed=seed, eps=eps, precision=prec, coulomb_k=coulomb_k,
                           real_space=1 if real_space else 0)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ctx = B.rbe2d_init(p, n_max, self.stream)
        self.P = P
        self.n_max = n_max
        self.params = dict(Lx=Lx, Ly=Ly, H=H, gamma_top=gamma_top, gamma_bot=gamma_bot, seed=seed)
        self.derived = B.rbe2d_get_derived(self.ctx)
        self._energy = torch.zeros(4, dtype=torch.float64, device=self.device)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.rbe2d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ batch
    def sample_k(self, step: int, return_k: bool = False):
        k = torch.empty((self.P, 3), dtype=torch.int32, device=self.device) if return_k else None
        B.rbe2d_sample_k(self.ctx, step, k)
        return k

    def set_k(self, k_idx):
        k = torch.as_tensor(k_idx, dtype=torch.int32).to(self.device).contiguous()
        if tuple(k.shape) != (self.P, 3):
            raise ValueError(f"k_idx must have shape ({self.P}, 3), got {tuple(k.shape)}")
        B.rbe2d_set_k(self.ctx, k)
        self._k_keep = k  # kept alive until the launch has consumed it

    # ------------------------------------------------------------------ inputs
    def _inputs(self, pos, q):
        # the kernels read these pointers as device memory of this context's GPU; host
        # arrays go through the binding's RBE2D_HOST_BUFFERS calls instead
        if pos.device != self.device or q.device != self.device:
            raise ValueError(f"pos and q must be tensors on {self.device}, got {pos.device} and {q.device}")
        if pos.dim() != 2 or pos.shape[1] != 3 or q.dim() != 1 or q.shape[0] != pos.shape[0]:
            raise ValueError(f"pos must be (N, 3) and q (N,), got {tuple(pos.shape)} and {tuple(q.shape)}")
        if pos.dtype == torch.float32:
            flags = B.RBE2D_INPUT_F32
            q = q.to(torch.float32)
        else:
            flags = 0
            pos = pos.to(torch.float64)
            q = q.to(torch.float64)
        return pos.contiguous(), q.contiguous(), flags

    def _out(self, out, N):
        """A caller's force array (contiguous (N, 3) of the output precision on this GPU),
        or a new one."""
        if out is None:
            return torch.empty((N, 3), dtype=self.out_dtype, device=self.device)
        if (out.device != self.device or out.dtype != self.out_dtype or tuple(out.shape) != (N, 3)
                or not out.is_contiguous()):
            raise ValueError(f"out must be a contiguous ({N}, 3) {self.out_dtype} tensor on {self.device}")
        return out

    def structure_factor(self, pos, q):
        pos, q, fl = self._inputs(pos, q)
        out = torch.empty((self.P, 4), dtype=torch.float64, device=self.device)
        B.rbe2d_structure_factor(self.ctx, q.shape[0], pos, q, fl, out)
        return out

    def force(self, pos, q, *, ibc=True, energy=False, potential=False, reuse_sf=False, validate=False,
              out=None):
        pos, q, fl = self._inputs(pos, q)
        N = q.shape[0]
        fl |= B.RBE2D_KSPACE
        if ibc:
            fl |= B.RBE2D_IBC
        if energy:
            fl |= B.RBE2D_ENERGY
        if potential:
            fl |= B.RBE2D_POTENTIAL
        if reuse_sf:
            fl |= B.RBE2D_REUSE_SF
        if validate:
            fl |= B.RBE2D_VALIDATE
        F = self._out(out, N)
        phi = torch.empty(N, dtype=self.out_dtype, device=self.device) if potential else None
        e = self._energy if energy else None
        B.rbe2d_force(self.ctx, N, pos, q, fl, F, phi, e)
        res = [F]
        if potential:
            res.append(phi)
        if energy:
            res.append(self._energy.clone())
        return res[0] if len(res) == 1 else tuple(res)

    def force_lattice(self, pos, q, nmax, *, ibc=True, energy=False, potential=False, out=None, accumulate=False):
        """Deterministic k-space sum over every k != 0 with |n_d| <= nmax[d] (the quantity
        the random batch estimates); same outputs as force()."""
        pos, q, fl = self._inputs(pos, q)
        N = q.shape[0]
        if ibc:
            fl |= B.RBE2D_IBC
        if energy:
            fl |= B.RBE2D_ENERGY
        if potential:
            fl |= B.RBE2D_POTENTIAL
        if accumulate:
            fl |= B.RBE2D_ACCUMULATE
        F = self._out(out, N)
        phi = torch.empty(N, dtype=self.out_dtype, device=self.device) if potential else None
        e = self._energy if energy else None
        B.rbe2d_force_lattice(self.ctx, N, pos, q, fl, nmax, F, phi, e)
        res = [F]
        if potential:
            res.append(phi)
        if energy:
            res.append(self._energy.clone())
        return res[0] if len(res) == 1 else tuple(res)

    def energy_backward(self, pos, q, grad_energy=1.0, *, reuse_sf=False):
        pos, q, fl = self._inputs(pos, q)
        N = q.shape[0]
        if reuse_sf:
            fl |= B.RBE2D_REUSE_SF
        dpos = torch.empty((N, 3), dtype=self.out_dtype, device=self.device)
        dq = torch.empty(N, dtype=self.out_dtype, device=self.device)
        dg = torch.empty(2, dtype=torch.float64, device=self.device)
        B.rbe2d_energy_backward(self.ctx, N, pos, q, fl, float(grad_energy), dpos, dq, dg)
        return dpos, dq, dg

    def sync_status(self):
        B.rbe2d_sync_status(self.ctx)


class RBE2DEnergy(torch.autograd.Function):
    """U = U_k + U_self + U_IBC of the current batch as a differentiable function of
    positions, charges and (gamma_top, gamma_bot).  Forward runs the structure factor
    and keeps only the P-sized results inside the context; backward runs the adjoint
    kernel, which recomputes the phases instead of storing the N x P table.  The
    gammas tensor must hold the context's contrasts (they are fixed at init)."""

    @staticmethod
    def forward(ctx_, model: RBE2D, pos, q, gammas):
        g = gammas.detach().to("cpu", torch.float64)
        if abs(float(g[0]) - model.params["gamma_top"]) > 0 or abs(float(g[1]) - model.params["gamma_bot"]) > 0:
            raise ValueError("gammas differ from the context's gamma_top / gamma_bot")
        F, e = model.force(pos.detach(), q.detach(), ibc=True, energy=True)
        ctx_.model = model
        ctx_.save_for_backward(pos.detach(), q.detach())
        ctx_.gdtype = gammas.dtype
        return (e[0] + e[1] + e[2]).to(pos.dtype)

    @staticmethod
    def backward(ctx_, grad):
        pos, q = ctx_.saved_tensors
        model = ctx_.model
        dpos, dq, dg = model.energy_backward(pos, q, float(grad), reuse_sf=True)
        return None, dpos.to(pos.dtype), dq.to(q.dtype), dg.to(ctx_.gdtype)
