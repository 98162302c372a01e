"""Host plumbing of the Omega split (several GPUs, one problem), on CPU ranks.

Two gloo ranks each take the bosonic range omega_partition gives them,
form their share of Eq. sd from the oracle's ladder kernel restricted to
those planes, and sum the shares with split.allreduce_sum: the sum must be
the oracle's full Sigma~ (the GPU kernels of each share are tested on one
GPU in tests/test_parity_gpu.py::test_omega_split_two_handles).
"""
import os

import numpy as np
import pytest

from paper_1507_00895_gb300 import split


@pytest.mark.parametrize("n_bos,world", [(1, 1), (15, 2), (15, 4), (7, 8), (31, 8), (3, 3)])
def test_omega_partition_covers_every_plane_once(n_bos, world):
    ranges = [split.omega_partition(n_bos, world, r) for r in range(world)]
    covered = [a for lo, hi in ranges for a in range(lo, hi)]
    assert covered == list(range(n_bos))
    sizes = [hi - lo for lo, hi in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_omega_partition_rejects_bad_arguments():
    with pytest.raises(ValueError):
        split.omega_partition(0, 2, 0)
    with pytest.raises(ValueError):
        split.omega_partition(5, 2, 2)


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    from oracle import df_oracle as O
    from paper_1507_00895_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = I.workload("square32_tp", nk=4, n_w=6, m_max=2)
        st = O.run_workload(w, n_iter=1)
        lo, hi = split.omega_partition(w.n_bos, world, rank)
        kern = np.zeros_like(st.kern)
        kern[lo:hi] = st.kern[lo:hi]
        part = O.dual_sigma_fft(kern, st.gt_ext, w.n_w, w.m_max, w.beta, w.dim, w.nk)
        t = torch.from_numpy(np.ascontiguousarray(part))
        split.allreduce_sum(t)
        if rank == 0:
            np.save(out_path, np.stack([t.numpy(), st.sigma]))
    finally:
        dist.destroy_process_group()


def test_omega_split_shares_sum_to_the_full_self_energy(tmp_path):
    import socket

    import torch.multiprocessing as tmp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = str(tmp_path / "sum.npy")
    tmp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    summed, full = np.load(out)
    assert np.max(np.abs(summed - full)) < 1e-13 * np.max(np.abs(full))
