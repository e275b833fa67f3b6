"""Tuner of the batched build (fp_build_batched).

Knobs that change the speed of a cloud's build but not its octree: the count
grid resolution g (any g <= s, g <= L_max; the node table, leaf grouping and
final layout are defined without it), the number of lanes the batch runs on,
whether the first two passes of all clouds are fused into one launch each,
and the fused count pass's block size and hot-cell table size (its
shared-memory privatisation depth).  The tuner times the candidates on the
device and keeps the fastest:
  - g per size bucket (floor(log2 n)), on a synthetic sample cloud of the
    bucket's size, each candidate built twice and timed once with CUDA events;
  - the lane count on the batch itself, each candidate timed as one call;
  - then, at that lane count, the fused first passes with every block size and
    table size, against the unfused batch.
The chunk threshold T stays as given (the octree does not depend on it either,
but chunk-size limits of the per-chunk scatter make T part of the workload).
"""
import math

import torch

from . import fastpoints as fp


def _time_ms(fn, stream):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        fn()
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def with_grid(prm, g):
    return fp.params(grid_log2=g, sub_log2=prm.sub_log2, max_level=prm.max_level, decim_modulus=prm.decim_modulus,
                     chunk_threshold=prm.chunk_threshold, node_capacity=prm.node_capacity)


def grid_candidates(prm, n):
    hi = min(7, prm.sub_log2, prm.max_level)
    # about 8..8^4 points per cell bracket the useful grids
    lo = max(1, min(hi, int(math.log(max(n, 8) / 4096.0, 8)) + 1))
    top = max(lo, min(hi, int(math.log(max(n, 8) / 8.0, 8)) + 1))
    return list(range(lo, top + 1))


class BatchTuner:
    def __init__(self, make_sample, stream=None):
        """make_sample(n) -> (n, 4) int32 CUDA tensor of a representative cloud."""
        self.make_sample = make_sample
        self.stream = stream or torch.cuda.current_stream()
        self.grid = {}      # (bucket, params key) -> g
        self.lanes = None
        self.log = []

    @staticmethod
    def _key(prm):
        return (prm.sub_log2, prm.max_level, prm.chunk_threshold, prm.node_capacity, prm.decim_modulus)

    def grid_for(self, n, prm):
        b = int(math.log2(max(n, 1)))
        k = (b, self._key(prm))
        if k not in self.grid:
            cands = grid_candidates(prm, n)
            if len(cands) == 1:
                self.grid[k] = cands[0]
            else:
                pts = self.make_sample(max(1, int(2 ** (b + 0.5))))
                best = None
                for g in cands:
                    p = with_grid(prm, g)
                    fp.build_octree(pts, p, stream=self.stream)   # warm (allocations, first launches)
                    ms = _time_ms(lambda: fp.build_octree(pts, p, stream=self.stream), self.stream)
                    self.log.append(("grid", b, g, ms))
                    if best is None or ms < best[0]:
                        best = (ms, g)
                self.grid[k] = best[1]
                del pts
        return self.grid[k]

    def tune_params(self, clouds):
        """clouds: list of (points, params) -> the same with g chosen per cloud."""
        return [(p, with_grid(prm, self.grid_for(p.shape[0], prm))) for p, prm in clouds]

    def tune_lanes(self, run, candidates=(4, 8, 16, 32)):
        """run(nlanes) enqueues the whole batch on self.stream; keeps the fastest."""
        best = None
        for L in candidates:
            run(L)   # warm
            ms = _time_ms(lambda: run(L), self.stream)
            self.log.append(("lanes", L, ms))
            if best is None or ms < best[0]:
                best = (ms, L)
        self.lanes = best[1]
        self.lanes_ms = best[0]
        return self.lanes

    def tune_opts(self, run, nlanes, variants=((256, 1024), (256, 4096), (512, 0), (512, 1024))):
        """run(opts) enqueues the whole batch with fp_build_batched_ex; returns the
        fastest fp_batch_opts at nlanes lanes, the unfused batch included."""
        cands = [fp.batch_opts(nlanes, 0, 256, 1024)] + [fp.batch_opts(nlanes, 1, t, s) for t, s in variants]
        best = None
        for o in cands:
            run(o)   # warm
            ms = _time_ms(lambda: run(o), self.stream)
            self.log.append(("opts", o.fused_first, o.count_threads, o.count_slots, ms))
            if best is None or ms < best[0]:
                best = (ms, o)
        self.opts = best[1]
        return self.opts
