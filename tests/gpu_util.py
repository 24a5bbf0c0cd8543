"""Helpers shared by the GPU parity tests (inputs and comparisons only)."""
import numpy as np
import torch

from oracle import mobility as om, rigid
from paper_1709_02410_gb300 import synth

DEV = "cuda:0"


def rel2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def handle_for(s, wall=True, kT=None):
    from paper_1709_02410_gb300 import Handle
    return Handle(synth.ETA, s.a, synth.KT if kT is None else kT, wall=wall)


def oracle_params(s, wall=True):
    return om.Params(synth.ETA, s.a, wall=wall)


def positions(s):
    """Oracle blob positions of a suspension (FP64 SoA)."""
    return rigid.blob_positions(s.q, s.theta, s.shape)
