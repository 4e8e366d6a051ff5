"""Host side of the row-partitioned DCGS2 (paper_2104_01253_gb300.partitioned) on CPU gloo
ranks: each rank's local CSR rows with re-based columns and its halo of w, assembled by
point-to-point messages, give exactly its rows of A w (Section 5's layout: rows of A and
of the vectors split across processes).  Includes a partition whose halo reaches past the
neighbouring rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _operator(N):
    from synth import convdiff_csr
    return convdiff_csr(N, 3, [1.0, 0.5, 0.25])


def _worker(rank, P, N, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=P)
    from paper_2104_01253_gb300 import partitioned as pt
    from synth import gaussian_vector
    Ah = _operator(N)
    blocks = pt.row_blocks(Ah.m, P)
    ranges = [pt.local_rows(Ah.row_ptr, Ah.col_idx, Ah.val, lo, hi)[3:] for lo, hi in blocks]
    plans = [pt.halo_plan(blocks, p, glo, ghi) for p, (glo, ghi) in enumerate(ranges)]
    lo, hi = blocks[rank]
    rp, ci, va, glo, ghi = pt.local_rows(Ah.row_ptr, Ah.col_idx, Ah.val, lo, hi)
    w = gaussian_vector(Ah.m, 7)
    w_ext = pt.halo_exchange(dist, blocks, rank, torch.as_tensor(w[lo:hi]), glo, ghi, plans)
    import scipy.sparse as sp
    Al = sp.csr_matrix((va, ci, rp), shape=(hi - lo, ghi - glo))
    out[rank] = (Al @ w_ext.numpy(), np.array_equal(w_ext.numpy(), w[glo:ghi]),
                 len(plans[rank]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("P,N", [(2, 9), (3, 9), (7, 5)])
def test_local_rows_and_halo_give_the_global_matvec(P, N):
    """(7, 5): m = 125 rows in blocks of 17-18 with a halo of 25 rows on each side, so an
    interior rank needs rows of two ranks on each side."""
    from paper_2104_01253_gb300 import partitioned as pt
    from synth import gaussian_vector
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(P, N, _free_port(), out), nprocs=P, join=True)
    Ah = _operator(N)
    ref = Ah.to_scipy() @ gaussian_vector(Ah.m, 7)
    for p, (lo, hi) in enumerate(pt.row_blocks(Ah.m, P)):
        y, halo_ok, _ = out[p]
        assert halo_ok
        assert np.array_equal(y, ref[lo:hi])
    if (P, N) == (7, 5):
        assert max(out[p][2] for p in range(P)) >= 3      # owners beyond the neighbours
