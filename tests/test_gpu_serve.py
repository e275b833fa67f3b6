"""The served request loop: every request's preview, node table and final
layout equal the oracle's, element by element, and are the same served alone,
served in a mix (admitted together, built on their own streams at the same
time, one of them out of core) and built by the plain calls."""
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_build_matches_oracle

pytestmark = pytest.mark.gpu

# kind, n, seed
REQS = [("lidar", 120_000, 51), ("uniform", 60_000, 52), ("lidar", 250_000, 53), ("uniform", 30_000, 54),
        ("lidar", 2_000_000, 55)]


def results_equal(a, b):
    for k in ("preview", "nodes", "final", "final_perm"):
        x, y = a[k].cpu().contiguous().view(torch.uint8), b[k].cpu().contiguous().view(torch.uint8)
        if x.shape != y.shape or not torch.equal(x, y):
            return k
    return None


def test_served_alone_mixed_plain(gpu_lib):
    from paper_2302_05002_gb300 import serve
    fp = gpu_lib
    prm = fp.params(grid_log2=6, sub_log2=7, max_level=15, decim_modulus=16, chunk_threshold=20_000,
                    node_capacity=2_000)
    hosts, wants = [], []
    oprm = oracle.params(prm.grid_log2, prm.sub_log2, prm.max_level, prm.decim_modulus, prm.chunk_threshold,
                         prm.node_capacity)
    for kind, n, seed in REQS:
        a = synth.uniform(n, seed) if kind == "uniform" else synth.lidar(n, seed)
        hosts.append(fp.as_points(a, "cuda").cpu().pin_memory())
        wants.append(oracle.build_all(a, oprm))
    needs = [serve.incore_need(h.shape[0], prm) for h in hosts]
    piece = 1 << 18
    # the out-of-core arena (half the budget) holds the largest request's minimum; the others fit in core
    budget = 2 * max(max(needs[:-1]), fp.ooc_arena_min(hosts[-1].shape[0], prm, piece)) + (1 << 20)
    assert needs[-1] > budget * 3 // 4, "the largest request must go out of core"

    # plain, in core
    plain = []
    for h in hosts:
        r = fp.build_octree(h.cuda(), prm)
        M = int(r["num_nodes"].item())
        k = int(r["preview_count"].item())
        plain.append(dict(preview=r["preview"][:k].cpu(), nodes=r["nodes"][:M].cpu(), final=r["final"].cpu(),
                          final_perm=r["final_perm"].cpu()))

    def serve_all(batch):
        srv = serve.Server(budget_bytes=budget, piece_points=piece)
        reqs = [serve.Request(i, hosts[i], prm) for i in batch]
        for r in reqs:
            srv.submit(r)
        srv.drain(len(reqs))
        srv.close()
        for r in reqs:
            assert r.error is None, r.error
            assert r.t_preview is not None and r.t_done is not None and r.t_preview <= r.t_done
        return {r.rid: r for r in reqs}, srv

    alone = {}
    for i in range(len(hosts)):
        got, _ = serve_all([i])
        alone[i] = got[i]
    mixed, srv = serve_all(list(range(len(hosts))))
    assert srv.peak_active >= 2, "requests were not built at the same time"
    assert alone[len(hosts) - 1].mode == "out-of-core"
    for i in range(len(hosts)):
        for got in (alone[i].result, mixed[i].result):
            assert_build_matches_oracle(wants[i], preview=got["preview"], nodes=got["nodes"], final=got["final"],
                                        final_perm=got["final_perm"])
        assert results_equal(alone[i].result, plain[i]) is None, (i, "alone", results_equal(alone[i].result, plain[i]))
        assert results_equal(mixed[i].result, plain[i]) is None, (i, "mixed", results_equal(mixed[i].result, plain[i]))
