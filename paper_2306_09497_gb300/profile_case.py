"""Small, self-contained launch of the hot kernels for profiling (ncu) on one GPU.

Runs `steps` fine IMEX steps of the T255 workload on S slices through the C ABI
(propagate_F), after one untimed warm-up step.  Sized to hold a few GB on the
device while every kernel's operands exceed the 129 MB L2.

    python -m paper_2306_09497_gb300.profile_case --M 255 --nlat 384 --nlon 768 --S 32 --steps 1 --prec fp64
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    import torch

    from paper_2306_09497_gb300 import inputs, swe

    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=255)
    ap.add_argument("--nlat", type=int, default=384)
    ap.add_argument("--nlon", type=int, default=768)
    ap.add_argument("--S", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--dt", type=float, default=432000.0 / 7296.0)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"])
    a = ap.parse_args()
    prec = swe.SWE_FP64 if a.prec == "fp64" else swe.SWE_SPLIT_BF16X3
    plan = swe.Plan(a.M, a.nlat, a.nlon, prec=prec)
    U = torch.from_numpy(inputs.random_state(a.M, a.S, seed=7).view(np.float64).copy()).cuda()
    out = torch.empty_like(U)
    plan.propagate(swe.stepper(swe.SWE_IMEX, a.dt, 1), U, out, a.S)       # warm-up (tables, factors)
    torch.cuda.synchronize()
    plan.propagate(swe.stepper(swe.SWE_IMEX, a.dt, a.steps), U, out, a.S)
    torch.cuda.synchronize()
    print("ok", float(out.abs().max()))


if __name__ == "__main__":
    main()
