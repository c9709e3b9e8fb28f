"""Moves a seeded synthetic group (``synth.Group``) onto the device as a GroupSpec.

Pure marshalling: dtype conversion and host-to-device copies of the model, the
observed data and the known weights; no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np
import torch

from .wri import C128, C64, GroupSpec


def to_device(grp, dtype: int = C64, device="cuda", source_free: bool = True, d=None, u=None,
              m=None) -> GroupSpec:
    """GroupSpec for ``grp`` (a synth.Group); ``d`` overrides grp.d, ``m`` overrides grp.m."""
    rdt = torch.float64 if dtype == C128 else torch.float32
    cdt = torch.complex128 if dtype == C128 else torch.complex64
    spec = grp.spec
    mm = grp.m if m is None else m
    dd = grp.d if d is None else d
    m_t = torch.as_tensor(np.ascontiguousarray(mm, dtype=np.float64).reshape(spec.shape), dtype=rdt).to(device)
    d_t = torch.as_tensor(np.ascontiguousarray(dd, dtype=np.complex128), dtype=cdt).to(device)
    al = None
    if not source_free:
        a = np.ascontiguousarray(grp.alpha, dtype=np.complex128)
        al = torch.view_as_real(torch.as_tensor(a)).contiguous().to(device)
    if u is None:
        u_t = torch.zeros(grp.nsys, spec.n, dtype=cdt, device=device)
    else:
        u_t = torch.as_tensor(np.ascontiguousarray(u), dtype=cdt).reshape(grp.nsys, spec.n).to(device)
    return GroupSpec(spec.nx, spec.ny, spec.nz, spec.npml, spec.h, grp.omega, grp.v_max, m_t,
                     np.asarray(grp.src, np.int64), np.asarray(grp.rec_off, np.int32),
                     np.asarray(grp.rec_idx, np.int32), d_t, grp.lam, u_t, al, grp.pml_R)
