"""Shared helpers of the GPU tests: run the CUDA path through the C ABI."""
from __future__ import annotations

import numpy as np


def as_device(a: np.ndarray):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def run_gpu(roi, lab, dims, N, M, xyz, offsets, where: str = "device", options: dict | None = None,
            chunks: int = 1, ctx=None):
    """C, C_end (int32 numpy) and stats from the library.  where: 'device'
    (torch CUDA tensors), 'host' (numpy) or 'pinned' (page-locked torch)."""
    import torch
    from paper_2302_09247_gb300 import fastcod as fc

    own = ctx is None
    if own:
        ctx = fc.Context(0)
    try:
        for k, v in (options or {}).items():
            ctx.set_option(k, v)
        if where == "device":
            ctx.set_volumes(as_device(roi), as_device(lab), dims, N, M)
        else:
            ctx.set_volumes(np.ascontiguousarray(roi), np.ascontiguousarray(lab), dims, N, M)
        ns = len(offsets) - 1
        bounds = np.linspace(0, ns, chunks + 1).astype(np.int64)
        for c in range(chunks):
            b, e = int(bounds[c]), int(bounds[c + 1])
            o = np.ascontiguousarray(offsets[b:e + 1] - offsets[b])
            x = np.ascontiguousarray(xyz[offsets[b]:offsets[e]])
            if where == "device":
                ctx.add_streamlines(as_device(x), as_device(o))
                torch.cuda.synchronize()
            elif where == "pinned":
                xp = torch.from_numpy(x).pin_memory()
                op = torch.from_numpy(o).pin_memory()
                ctx.add_streamlines(xp, op)
                ctx.sync()
            else:
                ctx.add_streamlines(x, o)
        C = ctx.connectivity()
        Ce = ctx.endpoint_connectivity()
        st = ctx.stats()
        return C, Ce, st
    finally:
        if own:
            ctx.close()
