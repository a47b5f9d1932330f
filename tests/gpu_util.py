"""Shared helpers of the GPU tests (no test functions here)."""
import numpy as np


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def mirror_oracle_frontier(F_orc, t_max, NEG_orc, NEG_gpu):
    """The oracle's f_t[i] (i = x - y) laid out as the GPU's L_t[d], d = -i."""
    G = F_orc[:, ::-1].copy()  # column i + T  ->  d + T with d = -i
    G[G == NEG_orc] = NEG_gpu
    return G.astype(np.int64)
