"""The sharded multi-GPU decode, simulated with gloo ranks on the CPU
(-m "not gpu"; no GPU is used).

Each rank takes its block-aligned output range (aceapex_shard_range),
computes the range's byte-level closure with the library's walk over the
match index (acx_debug_closure; the index comes from the oracle's parse),
decodes only that closure — literals, and the wanted matches byte-serially
in output order — and the ranks all-gather their ranges.  The assembled
output must equal the input: every rank's closure suffices on its own, with
no exchange before the gather."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, arc_path, data_path, result_path):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import oracle
    import paper_2608_10188_gb300 as acx
    from test_lib_cpu import _closure, _match_index

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    arc = open(arc_path, "rb").read()
    total = int(np.load(data_path).size)
    nb = (total + 16383) // 16384
    start, length = acx.shard_range(total, world, rank)
    idx = _match_index(arc, nb)
    need = _closure(acx, arc, idx, start, length) if length else {}
    out = np.zeros(total, np.uint8)
    for b in sorted(need):
        t, lit, B = oracle.parse_block(arc, b), oracle.block_stream(arc, b, 3), 16384 * b
        for ll, m, d, s, li in zip(t["ll"].tolist(), t["ml"].tolist(), t["dst"].tolist(), t["src"].tolist(),
                                   t["lit"].tolist()):
            out[d - ll:d] = lit[li:li + ll]
            if m and any(s0 < d - B + m and d - B < e0 for s0, e0 in need[b]):
                for j in range(m):
                    out[d + j] = out[s + j]
    mine = torch.from_numpy(out[start:start + length].copy())
    sizes = [acx.shard_range(total, world, r)[1] for r in range(world)]
    parts = [torch.zeros(n, dtype=torch.uint8) for n in sizes]
    # all_gather needs equal sizes: pad to the largest range
    m = max(sizes)
    padded = torch.zeros(m, dtype=torch.uint8)
    padded[:length] = mine
    gathered = [torch.zeros(m, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(gathered, padded)
    if rank == 0:
        whole = torch.cat([g[:n] for g, n in zip(gathered, sizes)]).numpy()
        np.save(result_path, whole)
        np.save(result_path.replace(".npy", "_closure.npy"), np.array([len(need)]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_decode_with_gloo_ranks(tmp_path, world):
    import torch.multiprocessing as mp

    import paper_2608_10188_gb300 as acx
    import synth
    acx.build.build()
    acx.load()
    data = synth.dna((1 << 20) + 4321, 17)
    arc = acx.encode(data)
    arc_path, data_path = str(tmp_path / "a.acx"), str(tmp_path / "d.npy")
    result_path = str(tmp_path / "out.npy")
    open(arc_path, "wb").write(arc)
    np.save(data_path, data)
    ranges = [acx.shard_range(data.size, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and sum(n for _, n in ranges) == data.size
    assert all(s % 16384 == 0 for s, _ in ranges)
    assert all(ranges[r][0] + ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    mp.start_processes(_rank_main, args=(world, _free_port(), arc_path, data_path, result_path), nprocs=world,
                       join=True, start_method="spawn")
    whole = np.load(result_path)
    assert np.array_equal(whole, data)
    # the last rank's closure reaches into earlier ranges (absolute offsets point back)
    assert int(np.load(result_path.replace(".npy", "_closure.npy"))[0]) > 0


def test_shard_range_edges():
    import paper_2608_10188_gb300 as acx
    acx.load()
    assert acx.shard_range(0, 4, 2) == (0, 0)
    assert acx.shard_range(100, 3, 0) == (0, 0) and acx.shard_range(100, 3, 2) == (0, 100)
    s = [acx.shard_range(5 * 16384 + 7, 2, r) for r in range(2)]
    assert s == [(0, 3 * 16384), (3 * 16384, 2 * 16384 + 7)]
    with pytest.raises(acx.AceapexError):
        acx.shard_range(100, 2, 2)
