"""Shared set-up of the GPU parity tests: the same seeded inputs for the library and the oracle."""
import numpy as np
import torch

import workloads as W
from oracle import assemble as OA, layout as OL, mesh as OM


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


class Case:
    """A macro mesh at a level with both the library mesh and the oracle space of one degree."""

    def __init__(self, meshname, level, degree):
        import paper_2404_08371_gb300 as hhg
        self.v, self.t = getattr(W, meshname)()
        self.level, self.degree = level, degree
        self.mesh = hhg.Mesh(self.v, self.t, level)
        self.S = OA.Space(OM.MacroMesh(self.v, self.t), level, degree)

    def packed(self, xg, dtype=torch.float64):
        return torch.tensor(OL.to_packed(self.S, xg), dtype=dtype, device="cuda")

    def unpack(self, y):
        yp = y.detach().cpu().double().numpy()
        return OL.from_packed(self.S, yp), OL.copies_spread(self.S, yp)
