"""Row-partitioned DCGS2 Arnoldi over several ranks (Section 5, Tables 1-2: the rows of A,
Q, w and v split across processes, one global sum of 2k + 2 numbers per step).

The per-rank GPU work is libkrylov's dcgs2_part_reduce / dcgs2_part_update /
dcgs2_part_finish; this module holds the host side a multi-rank caller needs:

  row_blocks      contiguous row ranges of P ranks (sizes differ by at most one);
  local_rows      a rank's rows of a CSR matrix, its column indices re-based onto the
                  contiguous range of w it reads (its own rows plus the halo);
  halo_exchange   that range of w assembled from the owning ranks with point-to-point
                  messages (torch.distributed, any backend);
  expansion       n steps and the CGS2 finish of one rank, given the halo exchange and
                  the global sum (dist.all_reduce on NCCL in production) as callables.

Every step of the arithmetic runs in the library's kernels; the callables only move data.
"""
from __future__ import annotations

import numpy as np


def row_blocks(m: int, P: int):
    """[(lo, hi)] of P contiguous row blocks covering 0..m-1."""
    b = [(m * p) // P for p in range(P + 1)]
    return list(zip(b[:-1], b[1:]))


def local_rows(row_ptr, col_idx, val, lo: int, hi: int):
    """Rows lo..hi-1 of a CSR matrix (numpy int32 / float64 arrays).  Returns (row_ptr,
    col_idx, val, glo, ghi): the local CSR whose column indices point into w[glo:ghi], the
    smallest contiguous range of w that covers the rank's own rows and every column its
    rows reach."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    a, b = int(rp[lo]), int(rp[hi])
    cols = np.asarray(col_idx[a:b], dtype=np.int64)
    glo = min(lo, int(cols.min())) if cols.size else lo
    ghi = max(hi, int(cols.max()) + 1) if cols.size else hi
    lrp = (rp[lo:hi + 1] - a).astype(np.int32)
    return lrp, (cols - glo).astype(np.int32), np.asarray(val[a:b], dtype=np.float64), glo, ghi


def halo_plan(blocks, rank: int, glo: int, ghi: int):
    """The pieces of w[glo:ghi] that other ranks own: [(owner, lo, hi)] in global rows."""
    out = []
    for p, (a, b) in enumerate(blocks):
        if p == rank:
            continue
        lo, hi = max(a, glo), min(b, ghi)
        if lo < hi:
            out.append((p, lo, hi))
    return out


def halo_exchange(dist, blocks, rank: int, w_local, glo: int, ghi: int, plans):
    """w[glo:ghi] on this rank from point-to-point messages.  plans[p] = halo_plan of rank p
    (every rank knows every plan, so each one sends exactly what the others need).  The
    tensors stay on w_local's device; with the gloo backend pass host tensors."""
    import torch
    lo_me, hi_me = blocks[rank]
    ops, recv = [], []
    for q, plan in enumerate(plans):
        if q == rank:
            continue
        for owner, lo, hi in plan:
            if owner == rank:                          # rank q needs rows lo..hi of mine
                ops.append(dist.P2POp(dist.isend, w_local[lo - lo_me:hi - lo_me].contiguous(), q))
    for owner, lo, hi in plans[rank]:
        buf = torch.empty(hi - lo, dtype=w_local.dtype, device=w_local.device)
        recv.append((lo, hi, buf))
        ops.append(dist.P2POp(dist.irecv, buf, owner))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    w_ext = torch.empty(ghi - glo, dtype=w_local.dtype, device=w_local.device)
    w_ext[lo_me - glo:hi_me - glo] = w_local
    for lo, hi, buf in recv:
        w_ext[lo - glo:hi - glo] = buf
    return w_ext


def expansion(kc, ctx, A_local, st, r0_local, n: int, exchange, allreduce):
    """n row-partitioned DCGS2 steps and the CGS2 finish on this rank.  exchange(w_local)
    returns the halo-extended w (device tensor, the range A_local's columns index);
    allreduce(t) returns the element-wise sum of the device tensor t over the ranks.  Makes
    n + 3 global sums in all: one per step, three for the finish."""
    import torch
    kc.dcgs2_arnoldi_init(ctx, A_local, st, r0_local)
    bufs = [torch.empty(2 * n + 2, dtype=torch.float64, device=st.w.device) for _ in range(2)]
    for k in range(n):
        part = bufs[k & 1][:2 * k + 2]
        kc.dcgs2_part_reduce(ctx, A_local, st, exchange(st.w[:st.m]), part)
        kc.dcgs2_part_update(ctx, A_local, st, allreduce(part))
    tot = None
    for phase, size in ((0, n + 1), (1, n + 1), (2, 1), (3, 0)):
        part = bufs[phase & 1][:size] if size else None
        kc.dcgs2_part_finish(ctx, A_local, st, phase, tot, part)
        tot = allreduce(part) if size else None
