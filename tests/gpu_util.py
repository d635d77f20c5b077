"""Helpers of the GPU parity tests: numpy <-> CUDA tensors and one-call runs
through the C-ABI binding."""
import numpy as np


def dev_u64(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def dev_u8(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def host_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def build(text_words: np.ndarray, n: int, sigma: int, layout: int = 0):
    from paper_2602_04103_gb300 import capi
    return capi.qr_build(dev_u64(text_words), n, sigma, layout=layout)


def rank(idx, q: np.ndarray, c):
    """rank(q, c) through qr_rank (int c) or qr_rank_c (array c)."""
    import torch
    from paper_2602_04103_gb300 import capi
    dq = dev_u64(q)
    out = torch.empty_like(dq)
    if isinstance(c, (int, np.integer)):
        capi.qr_rank(idx, dq, int(c), out)
    else:
        capi.qr_rank_c(idx, dq, dev_u8(c), out)
    return host_u64(out)


def rank4(idx, q: np.ndarray):
    import torch
    from paper_2602_04103_gb300 import capi
    dq = dev_u64(q)
    out = torch.empty((q.size, 4), dtype=torch.int64, device=dq.device)
    capi.qr_rank4(idx, dq, out)
    return host_u64(out).reshape(-1, 4)
