"""Straggler-time emulation (Section IV, Eq. (eqnTtotal)).

Every processor (cell) of the code finishes its coded product after a random
task time: a processor doing sigma_c long dot products has the exponential
distribution of rate mu stretched by sigma_c, T_c = sigma_c X_c (Section
IV-A).  The sink starts peeling as soon as the outputs received so far form a
decodable set, at

    T_par = min over decodable cell sets S of max_{c in S} T_c.

The emulation draws the times (the unscaled draws X_c are inputs, from
``workloads.exponential_draws``), sorts the arrivals, finds the first
decodable prefix with the library's online peel (``bpx_first_decodable``),
and runs the GPU path on exactly the cells that arrived by T_par (a cell-level
erasure mask: every later processor is a straggler).  T_par is model time (in
units of 1 / mu); the GPU times are measured.
"""
from __future__ import annotations

import numpy as np

from . import bpx


def task_times(code: "bpx.Code", X, scale_by_degree: bool = True) -> np.ndarray:
    """T_c = sigma_c X_c (sigma_c = the cell's degree), or X_c unscaled."""
    deg = np.diff(code.cell_ptr).astype(np.float64)
    X = np.asarray(X, dtype=np.float64)
    return X * deg if scale_by_degree else X.copy()


def arrivals(code: "bpx.Code", T):
    """(arrival order, number of arrivals to the first decodable set or -1,
    T_par or inf, sources recovered after each arrival)."""
    order = np.argsort(T, kind="stable").astype(np.int32)
    first, rec = bpx.first_decodable(code, order)
    t_par = float(T[order[first - 1]]) if first > 0 else float("inf")
    return order, first, t_par, rec


def emulate(code: "bpx.Code", A, B, h: int, precision: int, X, scale_by_degree: bool = True, ws=None,
            C=None, opts=None):
    """One emulated multiplication: task times from the draws X, the first
    decodable arrival set, and the GPU path on that set.  Returns a dict with
    T, order, first, t_par, the cell mask (1 = output not yet arrived), the
    decoded C and the device info words."""
    import torch
    T = task_times(code, X, scale_by_degree)
    order, first, t_par, rec = arrivals(code, T)
    mask = np.ones(code.num_cells, dtype=np.uint8)
    if first > 0:
        mask[order[:first]] = 0
    M, K = A.shape
    N = B.shape[1]
    if ws is None:
        ws = bpx.Workspace(code, M, N, K, h, precision, device=A.device)
    o = opts if opts is not None else bpx.default_opts()
    o.mask_cells = 1
    dmask = torch.from_numpy(mask).to(A.device)
    C, info = bpx.coded_matmul(code, A, B, h, precision, dmask, ws, C=C, opts=o)
    return dict(T=T, order=order, first=first, t_par=t_par, recovered_after=rec, cell_mask=mask, C=C, info=info)


def overlap_bound(code: "bpx.Code", order, first: int, peel_order, nchunks: int = 8):
    """How much of the peel could run while products still arrive.

    The first ``first`` cells of the arrival ``order`` (the decodable set)
    are cut into ``nchunks`` equal runs of arrivals.  A non-direct position
    of the peel plan (``peel_order``: rows (source, resolver, depth) in
    (depth, source) order, as ``bpx.schedule`` returns them) can be peeled
    once its resolver's product and every block it subtracts are there: its
    ready run is the latest of its resolver's run and the ready runs of the
    sources it subtracts (a direct source is ready with its resolver).
    Returns the count of non-direct positions per ready run: everything
    before the last run could overlap the products, the rest cannot."""
    order = np.asarray(order)
    po = np.asarray(peel_order)
    chunk = np.full(code.num_cells, -1, dtype=np.int64)
    if first > 0:
        chunk[order[:first]] = np.arange(first, dtype=np.int64) * nchunks // first
    ready = np.full(code.num_sources, -1, dtype=np.int64)
    counts = np.zeros(nchunks, dtype=np.int64)
    ptr, src = code.cell_ptr, code.cell_src
    for s, r, d in po:
        if s < 0:
            break
        rc = int(chunk[r])
        for t in src[ptr[r]:ptr[r + 1]]:
            if t != s:
                rc = max(rc, int(ready[t]))
        ready[s] = rc
        if d > 1:
            counts[rc] += 1
    return counts


def online_recovery(code: "bpx.Code", order, first: int, ws, nchunks: int = 8, device=None):
    """Sources the peel recovers from the arrivals so far, after each of the
    ``nchunks`` runs of the decodable set (the GPU schedule over each prefix:
    resolvers taken among the cells that have arrived)."""
    import torch
    out = []
    for j in range(nchunks):
        n_j = (j + 1) * first // nchunks
        mask = np.ones(code.num_cells, dtype=np.uint8)
        mask[np.asarray(order)[:n_j]] = 0
        _o, _r, info = bpx.schedule(code, torch.from_numpy(mask).to(device), ws, cells=True)
        out.append(int(info[bpx.INFO_RECOVERED].item()))
    return np.diff(np.asarray([0] + out, dtype=np.int64))
