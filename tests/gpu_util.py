"""Helpers shared by the GPU tests: numpy <-> CUDA tensors for unsigned data,
and the paper's permutation check (Sec. 4.1) evaluated per array on the GPU
with torch ops (modulus 2^31 - 1 so products fit int64)."""
import numpy as np

P31 = (1 << 31) - 1


def to_dev(a):
    import torch
    view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).to("cuda")


def to_host(t, dtype):
    return t.cpu().numpy().view(dtype)


def row_products(t, n, z=0x5BD1E995):
    """prod_i (z - a_i) mod (2^31 - 1) for every row of n keys (u32 or u64 data)."""
    import torch
    x = t.view(-1, n)
    if x.dtype == torch.int32:
        v = x.to(torch.int64) & 0xFFFFFFFF
        v = v % P31
    else:
        lo = x & 0xFFFFFFFF
        hi = (x >> 32) & 0xFFFFFFFF
        v = ((hi % P31) * ((1 << 32) % P31) + lo % P31) % P31
    acc = torch.ones(x.shape[0], dtype=torch.int64, device=x.device)
    for i in range(n):
        acc = (acc * ((z - v[:, i]) % P31)) % P31
    return acc


def rows_sorted(t, n):
    """True iff every row of n unsigned keys is non-decreasing."""
    import torch
    x = t.view(-1, n)
    if x.dtype == torch.int32:
        v = x.to(torch.int64) & 0xFFFFFFFF
        return bool((v[:, 1:] >= v[:, :-1]).all())
    # unsigned 64-bit order: flip the sign bit, then compare as signed
    v = x ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=x.device)
    return bool((v[:, 1:] >= v[:, :-1]).all())
