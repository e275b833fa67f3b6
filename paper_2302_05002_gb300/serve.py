"""Served builds: a request loop over clouds arriving in pinned host memory.

The paper's converter shows a preview at once and builds the octree behind it
(Sec. 3, Sec. 4.2).  Here many such requests share one GPU under a device
memory budget:
  - admission: a request is admitted as soon as its device need fits in the
    free budget (first fit in arrival order, an out-of-core request before
    in-core ones: it is long and bound by the host link, so in-core builds
    overlap it), so requests that arrive while others run are built alongside
    them (each on its own CUDA stream; their kernels overlap on the device).
    In-core builds of `big_points` or more fill most of the GPU and at most
    `big_slots` of them run at a time; smaller ones overlap freely; a request
    passed over `max_bypass` times blocks later admissions until it fits;
  - a cloud whose in-core need exceeds three quarters of the budget is built
    out of core (fp_build_ooc) in an arena of half the budget;
  - in-core requests stream their points in pieces with cudaMemcpyAsync on a
    side stream and decimate each piece as it lands, so the preview is back in
    pinned host memory before the octree is built; then the plain calls run;
  - an in-core request's octree (node table, final points and perm) stays on
    the device; an out-of-core one is written to pinned host memory (at most
    `ooc_slots` such requests at a time, each in its own host buffers,
    allocated when the server starts; one by default: an out-of-core build is
    bound by the host link, so a second one only shares the link while its
    arena keeps the other half of the budget from in-core requests);
  - per request: time to preview and time to the full octree (from arrival),
    both taken on the host when the device work is done.
Results do not depend on the mix: every request runs the same calls on its own
buffers.
"""
import collections
import threading
import time

import torch

from . import fastpoints as fp


class Request:
    def __init__(self, rid, host_pts, prm, preview_host=None):
        self.rid = rid
        self.host = host_pts            # (n, 4) int32, pinned
        self.n = host_pts.shape[0]
        self.prm = prm
        self.preview_host = preview_host   # optional pinned (slots, 4) int32 buffer for the streamed preview
        self.arrival = None
        self.t_admit = self.t_preview = self.t_done = None
        self.mode = None
        self.need = 0
        self.slot = None
        self.result = None
        self.error = None


def incore_need(n, prm):
    """Device bytes of an in-core request: points, outputs, workspace, grids, node table, preview."""
    cells = 1 << (3 * prm.grid_log2)
    ws = max(fp.workspace_size(k, n, prm) for k in ("bounds_decimate", "merge", "distribute", "octree",
                                                     "subsample"))
    ncap = fp.node_capacity_bound(n, prm)
    return (n * (16 + 16 + 4 + 4 + 16 + 4) + ws + cells * (4 + 16 + 4 + 8) + ncap * 40 +
            16 * fp._preview_cap(n, prm.decim_modulus) + (64 << 20))


def pick_request(queue, free, ooc_slot_free, big_points, big_active, big_slots=1, max_bypass=None):
    """The request the loop admits next, or None.  A request fits when its device
    need fits in the free budget and, out of core, a host slot is free, or, in
    core, it is smaller than big_points or fewer than big_slots such builds are
    running.  Of those, a waiting out-of-core request goes first (long and bound
    by the host link, so in-core builds overlap it), else the first in arrival
    order.  Aging: once the oldest waiting request has been passed over
    max_bypass times (requests behind it admitted while it did not fit), nothing
    else is admitted until it fits, so a large request cannot wait forever
    behind a stream of small ones."""
    if not queue:
        return None
    head = queue[0]

    def fits(r):
        return r.need <= free and (ooc_slot_free if r.mode == "out-of-core" else
                                   (r.n < big_points or big_active < big_slots))

    if max_bypass is not None and getattr(head, "bypassed", 0) >= max_bypass:
        return head if fits(head) else None
    ok = [r for r in queue if fits(r)]
    return next((r for r in ok if r.mode == "out-of-core"), ok[0] if ok else None)


def _preview_slot_cap(p, m):
    return fp._preview_cap(p, m)


def preview_slots_shape(n, piece, m):
    """Rows of the pinned preview buffer of an in-core request."""
    return max(1, (n + piece - 1) // piece) * _preview_slot_cap(piece, m), 4


class Server:
    def __init__(self, budget_bytes=24 << 30, piece_points=1 << 23, device=0, ooc_max_points=0, ooc_prm=None,
                 ooc_slots=1, big_points=1 << 24, big_slots=2, max_bypass=8):
        self.budget = budget_bytes
        self.big_points = big_points   # in-core builds this large fill the GPU: at most big_slots at a time
        self.big_slots = big_slots
        self.max_bypass = max_bypass   # aging bound of the admission (see pick_request)
        self.big_active = 0
        self.free = budget_bytes
        self.piece = piece_points
        self.ooc_slots = ooc_slots
        self.ooc_free = []   # pinned host store and outputs of every out-of-core slot (None: allocated per request)
        for _ in range(ooc_slots):
            self.ooc_free.append((torch.empty(fp.ooc_host_bytes(ooc_max_points, ooc_prm), dtype=torch.uint8)
                                  .pin_memory(), fp.ooc_outputs(ooc_max_points, ooc_prm)) if ooc_max_points else None)
        self.device = torch.device("cuda", device)
        self.cv = threading.Condition()
        self.queue = collections.deque()
        self.threads = []
        self.done = []
        self.peak_active = 0
        self.active = 0
        self._stop = False
        self._sched = threading.Thread(target=self._loop, daemon=True)
        self._sched.start()

    # ---- admission
    def submit(self, req):
        req.arrival = time.perf_counter()
        if incore_need(req.n, req.prm) <= self.budget * 3 // 4:
            req.mode, req.need = "in-core", incore_need(req.n, req.prm)
        else:
            req.mode, req.need = "out-of-core", self.budget // 2
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()

    def _loop(self):
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while True:
                    if self._stop and not self.queue:
                        return
                    pick = pick_request(self.queue, self.free, bool(self.ooc_free), self.big_points,
                                        self.big_active, self.big_slots, self.max_bypass)
                    if pick is not None:
                        break
                    self.cv.wait()
                for r in self.queue:   # passed over by a later arrival
                    if r is pick:
                        break
                    r.bypassed = getattr(r, "bypassed", 0) + 1
                self.queue.remove(pick)
                self.free -= pick.need
                if pick.mode == "out-of-core":
                    pick.slot = self.ooc_free.pop()
                elif pick.n >= self.big_points:
                    self.big_active += 1
                self.active += 1
                self.peak_active = max(self.peak_active, self.active)
            pick.t_admit = time.perf_counter()
            t = threading.Thread(target=self._work, args=(pick,), daemon=True)
            t.start()
            self.threads.append(t)

    def _release(self, req):
        with self.cv:
            self.free += req.need
            if req.mode == "out-of-core":
                self.ooc_free.append(req.slot)
            elif req.n >= self.big_points:
                self.big_active -= 1
            self.active -= 1
            self.done.append(req)
            self.cv.notify_all()

    def drain(self, count):
        """Wait until `count` requests are done; returns them in completion order."""
        with self.cv:
            while len(self.done) < count:
                self.cv.wait()
            return list(self.done)

    def close(self):
        with self.cv:
            self._stop = True
            self.cv.notify_all()
        self._sched.join()
        for t in self.threads:
            t.join()

    # ---- one request
    def _work(self, req):
        torch.cuda.set_device(self.device)
        try:
            if req.mode == "in-core":
                self._incore(req)
            else:
                self._ooc(req)
        except Exception as ex:   # reported on the request; the server keeps serving
            req.error = repr(ex)
        finally:
            self._release(req)

    def _ooc(self, req):
        arena = torch.empty(req.need, dtype=torch.uint8, device=self.device)
        st = torch.cuda.Stream(self.device)

        def on_preview():
            req.t_preview = time.perf_counter()

        scratch, out = req.slot if req.slot is not None and req.slot[1]["final"].shape[0] >= req.n else (None, None)
        if out is not None:   # the slot's outputs sized for the largest cloud: node capacity of this one
            out = dict(out, node_cap=fp.node_capacity_bound(req.n, req.prm),
                       preview_cap=fp._preview_cap(req.n, req.prm.decim_modulus))
        out = fp.build_ooc(req.host, req.prm, arena, piece_points=self.piece, scratch=scratch, out=out,
                           on_preview=on_preview, stream=st)
        req.t_done = time.perf_counter()
        k = int(out["preview_count"].item())
        req.result = dict(preview=out["preview"][:k], nodes=out["nodes"][: int(out["num_nodes"].item())],
                          final=out["final"][: req.n], final_perm=out["final_perm"][: req.n])
        del arena

    def _incore(self, req):
        n, prm, dev, P = req.n, req.prm, self.device, self.piece
        st, cs = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        L, S = fp.load(), fp._stream(st)
        pts = torch.empty((max(n, 1), 4), dtype=torch.int32, device=dev)
        out = fp.cloud_outputs(pts[:n], prm, leaf=False)
        ws_need = max(fp.workspace_size(k, n, prm) for k in ("bounds_decimate", "merge", "distribute", "octree",
                                                              "subsample"))
        ws = torch.empty(max(ws_need, 1), dtype=torch.uint8, device=dev)
        W, Wn = fp._ptr(ws), ws.numel()
        # pieces: copy on the side stream, decimate each as it lands
        npieces = (n + P - 1) // P
        pcap = _preview_slot_cap(P, prm.decim_modulus)
        slots = torch.empty((max(npieces, 1) * pcap, 4), dtype=torch.int32, device=dev)
        slot_n = torch.zeros(max(npieces, 1), dtype=torch.int64, device=dev)
        h_slots = req.preview_host if req.preview_host is not None else torch.empty_like(slots, device="cpu").pin_memory()
        h_slot_n = torch.empty_like(slot_n, device="cpu").pin_memory()
        for k in range(npieces):
            a, b = k * P, min(n, (k + 1) * P)
            with torch.cuda.stream(cs):
                pts[a:b].copy_(req.host[a:b], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cs)
            st.wait_event(ev)
            fp._check(L.fp_decimate(fp._ptr(pts[a:b]), b - a, a, prm.decim_modulus, fp._ptr(slots[k * pcap:]), pcap,
                                    fp._ptr(slot_n[k:]), W, Wn, S), "fp_decimate")
        with torch.cuda.stream(st):
            h_slots[: slots.shape[0]].copy_(slots, non_blocking=True)
            h_slot_n.copy_(slot_n, non_blocking=True)
            ev_prev = torch.cuda.Event()
            ev_prev.record(st)
        # the octree: the plain calls on the resident cloud; it stays on the device
        d = fp.cloud_desc(pts[:n], prm, out)
        fp.plain_calls(d, ws, stream=st)
        with torch.cuda.stream(st):
            ev_done = torch.cuda.Event()
            ev_done.record(st)
        ev_prev.synchronize()
        req.t_preview = time.perf_counter()
        ev_done.synchronize()
        req.t_done = time.perf_counter()
        counts = h_slot_n.tolist()
        prev = torch.cat([h_slots[k * pcap:k * pcap + int(c)] for k, c in enumerate(counts)]) if npieces else \
            torch.empty((0, 4), dtype=torch.int32)
        M = int(out["num_nodes"].item())
        req.result = dict(preview=prev, nodes=out["nodes"][:M], final=out["final"][:n],
                          final_perm=out["final_perm"][:n])
        del pts, ws, slots


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(xs) - 1)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)
