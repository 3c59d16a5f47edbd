"""Helpers shared by the GPU parity tests (no method arithmetic here)."""

import numpy as np
import torch


def dev(a, dtype=torch.int32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()
