"""Benchmark of the adaptive SpMV/SpMSpV hot path on GB300.

Default workload (one "step"): the x-density sweep on the FP32 27-point
stencil, 256^3 grid (16.8M rows, 449M entries, CSR and CSC resident): for
each density rho in {1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1}, one selector-driven
SpMSpV with x given as a list and the output as the structural list, and one
with x dense and y dense -- twelve products, each choosing its kernel on the
device. Metric: GB/s of work bytes (for every product, the fewest bytes any
correct candidate must touch: pointers, indices, values, gathered x and
written y) and its fraction of the measured HBM roofline.

Sections of the same line: the per-density table of the selected kernel
against every forced candidate (regret), the R-MAT scale-22 BFS + PageRank
step, whole BFS searches, incremental PageRank, handle creation, the batched
form (4096 Zipf-row vectors) and the backward form (16384^2 layer).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload stencil256|rmat22] [--sweep stencil256|rmat22]

--impl reference times the CPU oracle (the only other implementation of the
method; its multi-threaded form on every host core) on the same workload,
metric and unit. --sweep prints the per-kernel x-density table instead of the
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SpMV/SpMSpV GB/s and % HBM peak vs x density; batched & backward vs plain"
L2_FLUSH_BYTES = 512 << 20
KNAMES = ("pull_thread", "pull_warp", "pull_bal", "mpull_thread", "mpull_warp", "mpull_bal",
          "push_thread_atom", "push_warp_atom", "push_bal_atom", "push_thread_sort", "push_warp_sort",
          "push_bal_sort", "push_thread_priv", "push_warp_priv", "push_bal_priv")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ byte model
def useful_bytes(kid, m, n, nnz, nnz_x, nnz_s, nnz_y, s_v, s_x, s_y, x_sparse, sparse_out):
    """Bytes the selected candidate's pattern must touch (each element once)."""
    x_in = nnz_x * (4 + s_x) if x_sparse else n * s_x
    out = (nnz_y * (4 + s_y) + 8) if sparse_out else m * s_y
    if kid <= 2:  # pull SpMV: every row pointer, index and value, x, y
        return 4 * (m + 1) + nnz * (4 + s_v) + x_in + out
    if kid <= 5:  # validated pull: all indices, effective values, bitmap, listed x
        return 4 * (m + 1) + nnz * 4 + nnz_s * s_v + n / 8 + x_in + out
    # push: list, column pointer pairs, effective entries, output
    return x_in + 8 * nnz_x + nnz_s * (4 + s_v) + out


def work_bytes(m, n, nnz, nnz_x, nnz_s, nnz_y, s_v, s_x, s_y, x_sparse, sparse_out):
    """Work of one product, independent of the kernel that runs it: the least
    useful bytes any correct candidate (pull, validated pull, push) touches."""
    return min(useful_bytes(k, m, n, nnz, nnz_x, nnz_s, nnz_y, s_v, s_x, s_y, x_sparse, sparse_out)
               for k in (0, 3, 6))


LONG_ROW, LONG_SEG = 256, 4096  # the library's long-row split (rows > 256 entries, segments of 4096)


def long_row_launches(rowptr):
    """Extra launches of the thread and sub-warp pull kernels on a matrix with
    long rows: the warp-per-segment pass, plus its fix-up for rows of several
    segments."""
    deg = np.diff(rowptr)
    return int((deg > LONG_ROW).any()) + int((deg > LONG_SEG).any())


def direct_chain_launches(x_sparse, sparse_out):
    """Kernels of the warp push's direct chain (it runs beside the SWITCH node
    of every selector-driven call and returns at once unless chosen): x
    compaction for a dense x, the push, the write-out."""
    return (0 if x_sparse else 2) + 1 + (2 if sparse_out else 1)


def launches(kid, x_sparse, sparse_out, auto=True, long_extra=0, bool_fused=False):
    """Kernel launches of one call (mirrors the library's dispatch). The
    selector runs inside the feature pass and the SWITCH node launches no
    kernel of its own; a selector-driven call whose choice is not the warp
    push with atomics also launches that candidate's direct chain, whose
    kernels return at once. bool_fused: a Boolean list-output product on a
    matrix with long rows, whose thread pull runs the long rows' first chunks
    in its own launch (one extra launch: the second pass)."""
    c = 1  # feature pass
    compaction = 2  # block counts, write (each block sums the counts before it)
    scan = 2
    if auto and kid != 7:
        c += direct_chain_launches(x_sparse, sparse_out)
    if kid <= 5:
        dist = kid % 3
        if dist == 0 and bool_fused:
            c += 2
        else:
            c += (2 if dist == 2 else 1 + long_extra)
        if x_sparse:
            c += 2
        if sparse_out:
            c += compaction
        return c
    q = kid - 6
    dist, wb = q % 3, q // 3
    if not x_sparse:
        c += compaction
    if dist == 2 or wb != 0:
        c += 2  # list lengths + block sums, then their scan (and the balanced split's chunk owners)
    c += 1  # traversal
    if wb == 1:
        c += 3 * (1 + scan + 1) + 1  # radix passes (hist, scan, scatter) + reduce-by-key
    elif wb == 2:
        c += 1 + 1 + scan + 1 + 1 + 1  # memset, count, scan, copy, scatter, accumulate
    c += 1 if not sparse_out else compaction
    return c


# ------------------------------------------------------------------ measured DRAM traffic
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def sources_digest(files):
    """Digest of the library sources a traffic figure was taken with."""
    h = hashlib.sha256()
    for f in sorted(files):
        with open(os.path.join(ROOT, "paper_2006_16767_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def traffic_for(cls, model_bytes):
    """DRAM bytes per call of a call class, from one-kernel profiler captures
    of a smaller case of the same call, scaled by the byte model (the
    captures' traffic follows the model bytes); None when no capture covers
    the class or its kernels' sources changed since it was taken."""
    try:
        tab = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None, None
    e = tab.get("entries", {}).get(cls)
    if not e or sources_digest(e["sources"]) != e["sources_digest"]:
        return None, None
    scale = model_bytes / e["model_bytes_small"]
    return int(round(e["dram_bytes_small"] * scale)), {
        "captured_on": e["small_case"], "dram_bytes_small": e["dram_bytes_small"],
        "model_bytes_small": e["model_bytes_small"], "scale": round(scale, 4),
        "summary": e.get("summary")}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ workloads
def bfs_frontiers(rowptr, col, roots):
    """Successive BFS frontiers {v : level(v) = l} of each root, ascending.
    Levels come from scipy's BFS predecessor tree by pointer jumping."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    n = len(rowptr) - 1
    A = sp.csr_matrix((np.ones(len(col), np.int8), col, rowptr), shape=(n, n))
    out = []
    for root in roots:
        order, pred = breadth_first_order(A, root, directed=True, return_predecessors=True)
        anc = np.where(pred >= 0, pred, np.arange(n)).astype(np.int64)
        depth = (pred >= 0).astype(np.int64)
        while True:  # depth(v) += depth(anc(v)); anc(v) = anc(anc(v)) until every anc is a root
            nxt = anc[anc]
            if np.array_equal(nxt, anc):
                break
            depth = depth + depth[anc]
            anc = nxt
        level = np.full(n, -1, np.int64)
        level[order] = depth[order]
        for l in range(int(level.max()) + 1):
            out.append(np.flatnonzero(level == l).astype(np.int32))
    return out


class Stencil256:
    """FP32 27-point stencil on a side^3 grid; one product per (density, x
    format): x as a list with the structural output list, and x dense with a
    dense y."""
    name = "stencil256_density_sweep"
    RHOS = (1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0)
    dtype = "f32"

    def __init__(self, side=256):
        import gen
        self.side = side
        t = time.time()
        self.rowptr, self.col, self.val, self.rowsum = gen.stencil27(side, gen.config_seed(5))
        self.gen_s = time.time() - t
        self.m = self.n = side ** 3
        self.nnz = len(self.col)
        self.colcount = np.bincount(self.col, minlength=self.n)
        self.xs = []
        for rho in self.RHOS:
            k = max(1, int(round(rho * self.n)))
            idx, val = gen.sparse_x(self.n, k, gen.config_seed(5), 11, np.float32)
            self.xs.append((rho, idx, val, int(self.colcount[idx].sum())))
        # call order of a step: ascending density, the list form then the dense form
        self.plan = [(i, fmt) for i in range(len(self.RHOS)) for fmt in ("list", "dense")]

    @staticmethod
    def label(rho, fmt):
        return f"{fmt}:{rho:g}"

    def setup_gpu(self, asv, torch, dev):
        self.asv, self.torch = asv, torch
        m, n = self.m, self.n
        self.rp_d = torch.from_numpy(self.rowptr).to(dev)
        self.col_d = torch.from_numpy(self.col).to(dev)
        self.val_d = torch.from_numpy(self.val).to(dev)
        self.A = asv.Matrix(m, n, self.rp_d, self.col_d, self.val_d)
        self.idx_d, self.xval_d, self.xd_d = [], [], []
        for rho, idx, val, _ in self.xs:
            it = torch.from_numpy(idx).to(dev)
            vt = torch.from_numpy(val).to(dev)
            xd = torch.zeros(n, dtype=torch.float32, device=dev)
            xd[it.long()] = vt
            self.idx_d.append(it)
            self.xval_d.append(vt)
            self.xd_d.append(xd)
        nr = len(self.RHOS)
        self.cnt_d = torch.tensor([[len(x[1])] for x in self.xs], dtype=torch.int64, device=dev)
        self.nnz_y = torch.zeros(nr, dtype=torch.int64, device=dev)
        self.yidx = [torch.empty(m, dtype=torch.int32, device=dev) for _ in range(nr)]
        self.yval = [torch.empty(m, dtype=torch.float32, device=dev) for _ in range(nr)]
        self.yd = [torch.empty(m, dtype=torch.float32, device=dev) for _ in range(nr)]
        self.calls = []
        for i, fmt in self.plan:
            rho = self.RHOS[i]
            if fmt == "list":
                kid, vf = asv.asv_select(self.A.handle, self.cnt_d[i], self.idx_d[i], self.xval_d[i],
                                         out_mode=asv.ASV_OUT_SPARSE)
            else:
                kid, vf = asv.asv_select(self.A.handle, x_dense=self.xd_d[i])
            self.calls.append(dict(kind=self.label(rho, fmt), kid=kid, nnz_x=vf["nnz_x"], nnz_s=vf["nnz_s"],
                                   fmt=fmt, i=i))
        self.run_step()
        torch.cuda.synchronize()
        ny = self.nnz_y.cpu().numpy()
        for c in self.calls:
            sparse = c["fmt"] == "list"
            c["nnz_y"] = int(ny[c["i"]]) if sparse else m
            args_ = (m, n, self.nnz, c["nnz_x"], c["nnz_s"], c["nnz_y"], 4, 4, 4, sparse, sparse)
            c["bytes"] = work_bytes(*args_)
            c["kbytes"] = useful_bytes(c["kid"], *args_)
            c["launches"] = launches(c["kid"], sparse, sparse)

    def call(self, c, kernel="auto", xidx=None, xval=None, xd=None, cnt=None):
        asv, i = self.asv, c["i"]
        xidx = self.idx_d[i] if xidx is None else xidx
        xval = self.xval_d[i] if xval is None else xval
        cnt = self.cnt_d[i] if cnt is None else cnt
        if c["fmt"] == "list":
            asv.asv_spmspv(self.A.handle, cnt, xidx, xval, None, asv.ASV_OUT_SPARSE, None, self.yidx[i],
                           self.yval[i], self.nnz_y[i:i + 1], self.m, kernel)
        else:
            asv.asv_spmspv(self.A.handle, None, None, None, self.xd_d[i] if xd is None else xd,
                           asv.ASV_OUT_DENSE, self.yd[i], kernel=kernel)

    def run_step(self, events=None, direct=False):
        """One step; direct=True replays the selector's recorded choices as
        direct launches (for the profiler, which does not see kernels inside
        conditional graph nodes); the timed steps always run the selector."""
        nvtx = self.torch.cuda.nvtx if direct else None
        for j, c in enumerate(self.calls):
            if events is not None:
                events[j][0].record()
            if nvtx:
                nvtx.range_push(f"{c['kind']}:{KNAMES[c['kid']]}")
            self.call(c, c["kid"] if direct else "auto")
            if nvtx:
                nvtx.range_pop()
            if events is not None:
                events[j][1].record()

    # end to end through the public API: inputs from pinned host memory, the
    # step's results (lists of the exact size the device reports, dense y) back
    def e2e_setup(self, torch):
        self.h_idx = [torch.from_numpy(x[1]).pin_memory() for x in self.xs]
        self.h_val = [torch.from_numpy(x[2]).pin_memory() for x in self.xs]
        self.h_cnt = self.cnt_d.cpu().pin_memory()
        self.h_xd = [x.cpu().pin_memory() for x in self.xd_d]
        self.d_idx = [torch.empty_like(t) for t in self.idx_d]
        self.d_val = [torch.empty_like(t) for t in self.xval_d]
        self.d_cnt = torch.empty_like(self.cnt_d)
        self.d_xd = [torch.empty_like(t) for t in self.xd_d]
        self.h_nnzy = torch.empty(len(self.RHOS), dtype=torch.int64).pin_memory()
        self.h_yidx = [torch.empty(self.m, dtype=torch.int32).pin_memory() for _ in self.RHOS]
        self.h_yval = [torch.empty(self.m, dtype=torch.float32).pin_memory() for _ in self.RHOS]
        self.h_yd = [torch.empty(self.m, dtype=torch.float32).pin_memory() for _ in self.RHOS]
        h2d = sum(t.numel() * 4 for t in self.h_idx + self.h_val + self.h_xd) + self.h_cnt.numel() * 8
        d2h = sum(8 + c["nnz_y"] * 8 for c in self.calls if c["fmt"] == "list") + \
            sum(self.m * 4 for c in self.calls if c["fmt"] == "dense")
        return h2d, d2h

    def e2e_step(self):
        """One step through the public API with its copies: every call's input
        goes host -> device on a copy stream and the call waits only for its
        own input, so later inputs cross the link while earlier products run;
        every dense output goes back on a second copy stream as soon as its
        product is done; a list output, whose size only the device knows, goes
        back on a third as soon as its count (read on a fourth) reaches the
        host, while the later products run."""
        torch = self.torch
        cur = torch.cuda.current_stream()
        if not hasattr(self, "s_in"):
            self.s_in, self.s_out, self.s_cnt, self.s_list = (torch.cuda.Stream() for _ in range(4))
            self.ev_in = [torch.cuda.Event() for _ in self.calls]
            self.ev_done = [torch.cuda.Event() for _ in self.calls]
            self.ev_cnt = [torch.cuda.Event() for _ in self.calls]
        for st in (self.s_in, self.s_out, self.s_cnt, self.s_list):
            st.wait_stream(cur)
        with torch.cuda.stream(self.s_in):
            self.d_cnt.copy_(self.h_cnt, non_blocking=True)
            for j, c in enumerate(self.calls):
                i = c["i"]
                if c["fmt"] == "list":
                    self.d_idx[i].copy_(self.h_idx[i], non_blocking=True)
                    self.d_val[i].copy_(self.h_val[i], non_blocking=True)
                else:
                    self.d_xd[i].copy_(self.h_xd[i], non_blocking=True)
                self.ev_in[j].record(self.s_in)
        for j, c in enumerate(self.calls):
            i = c["i"]
            cur.wait_event(self.ev_in[j])
            self.call(c, "auto", self.d_idx[i], self.d_val[i], self.d_xd[i], self.d_cnt[i])
            self.ev_done[j].record(cur)
            if c["fmt"] == "dense":
                self.s_out.wait_event(self.ev_done[j])
                with torch.cuda.stream(self.s_out):
                    self.h_yd[i].copy_(self.yd[i], non_blocking=True)
            else:
                self.s_cnt.wait_event(self.ev_done[j])
                with torch.cuda.stream(self.s_cnt):
                    self.h_nnzy[i:i + 1].copy_(self.nnz_y[i:i + 1], non_blocking=True)
                    self.ev_cnt[j].record(self.s_cnt)
        for j, c in enumerate(self.calls):
            if c["fmt"] == "list":
                self.ev_cnt[j].synchronize()  # this list's size decides its copy
                i = c["i"]
                k = int(self.h_nnzy[i])
                with torch.cuda.stream(self.s_list):
                    self.h_yidx[i][:k].copy_(self.yidx[i][:k], non_blocking=True)
                    self.h_yval[i][:k].copy_(self.yval[i][:k], non_blocking=True)
        cur.wait_stream(self.s_out)
        cur.wait_stream(self.s_list)

    def config(self):
        return {"workload": self.name, "matrix": f"27-point stencil {self.side}^3, FP32, CSR + CSC resident",
                "m": self.m, "nnz": self.nnz, "x_densities": list(self.RHOS),
                "calls_per_step": len(self.calls),
                "formats": "per density: x list -> y list (SpMSpV), x dense -> y dense",
                "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)", "seed": 20061681}

    # the oracle on the same products (CPU baseline): the row-major product
    # for a dense x, and for a list the oracle routine whose pattern touches
    # fewer bytes (column-major push when the listed columns are short)
    def oracle_prepare(self):
        import oracle
        if getattr(self, "_oracle_ready", False):
            return
        self.val64 = self.val.astype(np.float64)
        self.colptr, self.rowidx, perm = oracle.csr_to_csc(self.m, self.n, self.rowptr, self.col)
        self.val64_csc = self.val64[perm]
        self.x64 = [(x[1], x[2].astype(np.float64)) for x in self.xs]
        self.xd64 = [gen_dense(self.n, x[1], x[2]) for x in self.xs]
        self._oracle_ready = True

    def oracle_step(self, par):
        import oracle
        self.oracle_prepare()
        t = time.perf_counter()
        for c in self.calls:
            i = c["i"]
            if c["fmt"] == "dense":
                (oracle.csr_pull_par if par else oracle.csr_pull)(self.rowptr, self.col, self.val64, self.xd64[i])
            elif c["nnz_s"] * 8 < self.nnz * 4:
                (oracle.csc_push_par if par else oracle.csc_push)(self.m, self.colptr, self.rowidx, self.val64_csc,
                                                                   *self.x64[i])
            else:
                (oracle.spmspv_rowmajor_par if par else oracle.spmspv_rowmajor)(self.n, self.rowptr, self.col,
                                                                                 self.val64, *self.x64[i])
        return sum(c["bytes"] for c in self.calls), time.perf_counter() - t

    def plan_calls_host(self):
        """The step's calls with their byte model from the oracle alone (no
        GPU), for the reference arm: the selected kernel does not enter the
        work bytes."""
        import oracle
        self.oracle_prepare()
        self.calls = []
        for i, fmt in self.plan:
            rho, idx, val, nnz_s = self.xs[i]
            sparse = fmt == "list"
            nnz_y = self.m
            if sparse:  # the structural output set: rows with an entry in a listed column
                nnz_y = int(oracle.csc_push(self.m, self.colptr, self.rowidx, None, idx, None)[1].sum())
            b = work_bytes(self.m, self.n, self.nnz, len(idx), nnz_s, nnz_y, 4, 4, 4, sparse, sparse)
            self.calls.append(dict(kind=self.label(rho, fmt), fmt=fmt, i=i, nnz_x=len(idx), nnz_s=nnz_s,
                                   nnz_y=nnz_y, bytes=b))


def gen_dense(n, idx, val):
    import gen
    return gen.densify(n, idx, np.asarray(val, np.float64))


class Rmat22:
    """R-MAT scale 22 BFS frontiers (Boolean) + one FP32 PageRank step."""
    name = "rmat22_bfs8_pagerank"
    dtype = "u8 (OR,AND) + f32"

    def __init__(self, scale=22, edge_factor=16, roots=8):
        import gen
        self.scale, self.edge_factor, self.nroots = scale, edge_factor, roots
        t = time.time()
        self.rowptr, self.col = gen.rmat(scale, edge_factor, gen.config_seed(2))
        self.gen_s = time.time() - t
        self.n = self.m = 1 << scale
        self.nnz = len(self.col)
        self.long_extra = long_row_launches(self.rowptr)
        # a Boolean list output: the long-row pass and its second pass, no fix-up
        self.long_extra_flags = 2 if self.long_extra else 0
        deg = np.diff(self.rowptr)
        cand = np.flatnonzero(deg > 0)
        pick = gen.randint(roots, len(cand), gen.config_seed(2), stream=7)
        self.roots = [int(cand[i]) for i in pick]
        r = gen.uniform(self.n, 0.0, 1.0, gen.config_seed(2), stream=8)
        r /= r.sum()
        self.pr_x = np.where(deg > 0, r / np.maximum(deg, 1), 0.0).astype(np.float32)

    def setup_gpu(self, asv, torch, dev):
        self.torch = torch
        self.rp_d = torch.from_numpy(self.rowptr).to(dev)
        self.col_d = torch.from_numpy(self.col).to(dev)
        self.ones_d = torch.ones(self.nnz, dtype=torch.float32, device=dev)
        self.Ab = asv.Matrix(self.m, self.n, self.rp_d, self.col_d, None)
        self.Af = asv.Matrix(self.m, self.n, self.rp_d, self.col_d, self.ones_d)
        self.x_pr = torch.from_numpy(self.pr_x).to(dev)
        self.y_pr = torch.empty(self.m, dtype=torch.float32, device=dev)
        # BFS frontiers (inputs, prepared on the host with scipy's BFS)
        self.frontiers_host = bfs_frontiers(self.rowptr, self.col, self.roots)
        self.frontiers = [torch.from_numpy(f).to(dev) for f in self.frontiers_host]
        nf = len(self.frontiers)
        self.counts = torch.tensor([[f.numel()] for f in self.frontiers], dtype=torch.int64, device=dev)
        self.nnz_y = torch.zeros(nf + 1, dtype=torch.int64, device=dev)
        # every level product keeps its own output list (the e2e leg reads them all back)
        self.yidx = [torch.empty(self.m, dtype=torch.int32, device=dev) for _ in range(nf)]
        self.calls = []
        for i, f in enumerate(self.frontiers):
            kid, vf = asv.asv_select(self.Ab.handle, self.counts[i], f, out_mode=asv.ASV_OUT_SPARSE)
            self.calls.append(dict(kind="bfs", kid=kid, nnz_x=vf["nnz_x"], nnz_s=vf["nnz_s"]))
        kid, vf = asv.asv_select(self.Af.handle, x_dense=self.x_pr)
        self.calls.append(dict(kind="pagerank", kid=kid, nnz_x=vf["nnz_x"], nnz_s=vf["nnz_s"]))
        self.asv = asv
        self.run_step()
        torch.cuda.synchronize()
        ny = self.nnz_y.cpu().numpy()
        for i, c in enumerate(self.calls):
            if c["kind"] == "bfs":
                c["nnz_y"] = int(ny[i])
                args_ = (self.m, self.n, self.nnz, c["nnz_x"], c["nnz_s"], c["nnz_y"], 0, 0, 0, True, True)
                c["bytes"] = work_bytes(*args_)
                c["kbytes"] = useful_bytes(c["kid"], *args_)
                c["launches"] = launches(c["kid"], True, True, long_extra=self.long_extra_flags,
                                         bool_fused=bool(self.long_extra))
            else:
                c["nnz_y"] = self.m
                args_ = (self.m, self.n, self.nnz, c["nnz_x"], c["nnz_s"], self.m, 4, 4, 4, False, False)
                c["bytes"] = work_bytes(*args_)
                c["kbytes"] = useful_bytes(c["kid"], *args_)
                c["launches"] = launches(c["kid"], False, False, long_extra=self.long_extra)

    def run_step(self, events=None, direct=False, fronts=None, counts=None, x_pr=None):
        """One step. direct=True replays the selector's recorded choices as
        direct launches (the profiler cannot see kernels inside graphs with
        conditional nodes); the timed steps always run the selector."""
        asv = self.asv
        h = self.Ab.handle
        fronts = self.frontiers if fronts is None else fronts
        counts = self.counts if counts is None else counts
        nvtx = self.torch.cuda.nvtx if direct else None  # per-call ranges for the profiler's launch list
        for i, f in enumerate(fronts):
            if events is not None:
                events[i][0].record()
            k = self.calls[i]["kid"] if direct else "auto"
            if nvtx:
                nvtx.range_push(f"bfs:{KNAMES[k]}")
            asv.asv_spmspv(h, counts[i], f, None, None, asv.ASV_OUT_SPARSE, None, self.yidx[i], None,
                           self.nnz_y[i:i + 1], self.m, k)
            if nvtx:
                nvtx.range_pop()
            if events is not None:
                events[i][1].record()
        j = len(fronts)
        if events is not None:
            events[j][0].record()
        if nvtx:
            nvtx.range_push(f"pagerank:{KNAMES[self.calls[j]['kid']]}")
        asv.asv_spmv(self.Af.handle, self.x_pr if x_pr is None else x_pr, self.y_pr,
                     self.calls[j]["kid"] if direct else "auto")
        if nvtx:
            nvtx.range_pop()
        if events is not None:
            events[j][1].record()

    def e2e_setup(self, torch):
        self.h_front = [f.cpu().pin_memory() for f in self.frontiers]
        self.h_counts = self.counts.cpu().pin_memory()
        self.h_prx = torch.from_numpy(self.pr_x).pin_memory()
        self.h_ypr = torch.empty(self.m, dtype=torch.float32).pin_memory()
        self.h_nnzy = torch.empty(len(self.frontiers) + 1, dtype=torch.int64).pin_memory()
        self.h_yidx = [torch.empty(self.m, dtype=torch.int32).pin_memory() for _ in self.frontiers]
        self.d_front = [torch.empty_like(f) for f in self.frontiers]
        self.d_counts = torch.empty_like(self.counts)
        self.d_prx = torch.empty_like(self.x_pr)
        h2d = sum(f.numel() * 4 for f in self.h_front) + self.h_counts.numel() * 8 + self.h_prx.numel() * 4
        d2h = self.h_ypr.numel() * 4 + sum(8 + c["nnz_y"] * 4 for c in self.calls if c["kind"] == "bfs")
        return h2d, d2h

    def e2e_step(self):
        """One step through the public API with its copies: the counts and then
        every frontier go host -> device on a copy stream, each product waiting
        only for its own input; each new frontier goes back on another copy
        stream as soon as its size (read on a third) reaches the host, and the
        PageRank y on a fourth, while the later products run."""
        torch = self.torch
        asv = self.asv
        cur = torch.cuda.current_stream()
        nf = len(self.frontiers)
        if not hasattr(self, "s_in"):
            self.s_in, self.s_out, self.s_cnt, self.s_list = (torch.cuda.Stream() for _ in range(4))
            self.ev_in = [torch.cuda.Event() for _ in range(nf + 1)]
            self.ev_done = [torch.cuda.Event() for _ in range(nf + 1)]
            self.ev_cnt = [torch.cuda.Event() for _ in range(nf)]
        for st in (self.s_in, self.s_out, self.s_cnt, self.s_list):
            st.wait_stream(cur)
        with torch.cuda.stream(self.s_in):
            self.d_counts.copy_(self.h_counts, non_blocking=True)
            for i, (hf, df) in enumerate(zip(self.h_front, self.d_front)):
                df.copy_(hf, non_blocking=True)
                self.ev_in[i].record(self.s_in)
            self.d_prx.copy_(self.h_prx, non_blocking=True)
            self.ev_in[nf].record(self.s_in)
        h = self.Ab.handle
        for i in range(nf):
            cur.wait_event(self.ev_in[i])
            asv.asv_spmspv(h, self.d_counts[i], self.d_front[i], None, None, asv.ASV_OUT_SPARSE, None, self.yidx[i],
                           None, self.nnz_y[i:i + 1], self.m, "auto")
            self.ev_done[i].record(cur)
            self.s_cnt.wait_event(self.ev_done[i])
            with torch.cuda.stream(self.s_cnt):
                self.h_nnzy[i:i + 1].copy_(self.nnz_y[i:i + 1], non_blocking=True)
                self.ev_cnt[i].record(self.s_cnt)
        cur.wait_event(self.ev_in[nf])
        asv.asv_spmv(self.Af.handle, self.d_prx, self.y_pr, "auto")
        self.ev_done[nf].record(cur)
        self.s_out.wait_event(self.ev_done[nf])
        with torch.cuda.stream(self.s_out):
            self.h_ypr.copy_(self.y_pr, non_blocking=True)
        for i in range(nf):
            self.ev_cnt[i].synchronize()  # this frontier's size decides its copy
            k = int(self.h_nnzy[i])
            with torch.cuda.stream(self.s_list):
                self.h_yidx[i][:k].copy_(self.yidx[i][:k], non_blocking=True)
        cur.wait_stream(self.s_out)
        cur.wait_stream(self.s_list)

    def config(self):
        return {"workload": self.name, "graph": f"rmat scale {self.scale} edge factor {self.edge_factor}",
                "n": self.n, "nnz": self.nnz, "roots": self.nroots, "bfs_levels": len(self.frontiers_host),
                "calls_per_step": len(self.calls), "bfs_output": "sparse list", "pagerank": "fp32 dense x",
                "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)", "seed": 20061678}

    def oracle_step(self, par, max_bfs_calls=None):
        import oracle
        xs = self.pr_x.astype(np.float64)
        nb = len(self.calls) - 1 if max_bfs_calls is None else min(max_bfs_calls, len(self.calls) - 1)
        t_tot, b_tot = 0.0, 0.0
        t = time.perf_counter()
        (oracle.csr_pull_par if par else oracle.csr_pull)(self.rowptr, self.col, None, xs)
        t_tot += time.perf_counter() - t
        b_tot += self.calls[-1]["bytes"]
        for i in range(nb):
            xb = np.zeros(self.n, np.uint8)
            xb[self.frontiers_host[i]] = 1
            t = time.perf_counter()
            oracle.bool_pull(self.rowptr, self.col, xb)
            t_tot += time.perf_counter() - t
            b_tot += self.calls[i]["bytes"]
        return b_tot, t_tot


def _time(torch, fn, reps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure(W, torch, dev, steps, warmup, direct=False, world=1, dist=None, clocks_index=None):
    """Times `steps` steps of workload W (CUDA events on the launching stream,
    L2 flushed before each step) and the same step end to end through the
    public API; returns the figures of the JSON line."""
    asv = W.asv
    hbm, peak_kind = peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ncalls = len(W.calls)
    for _ in range(max(3, warmup)):
        flush.zero_()
        W.run_step(direct=direct)
    torch.cuda.synchronize()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    call_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ncalls)]
               for _ in range(steps)]
    clocks = ClockSampler(clocks_index) if clocks_index is not None else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    t_wall = time.perf_counter()
    for s in range(steps):
        flush.zero_()
        torch.cuda.nvtx.range_push("timed_step")
        step_ev[s][0].record()
        W.run_step(call_ev[s], direct=direct)
        step_ev[s][1].record()
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clk = None
    if clocks:
        time.sleep(0.2)
        clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in step_ev) / steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    step_bytes = sum(c["bytes"] for c in W.calls)
    value = step_bytes * world / (ms * 1e-3) / 1e9

    # per call class (kind, selected kernel): durations from the per-call
    # events, recorded on the stream the calls are launched on
    per_k = {}
    for s in range(steps):
        for i, c in enumerate(W.calls):
            d = call_ev[s][i][0].elapsed_time(call_ev[s][i][1])
            e = per_k.setdefault((c["kind"], c["kid"]), {"ms": 0.0, "bytes": 0.0, "n": 0})
            e["ms"] += d
            e["bytes"] += c["kbytes"]
            e["n"] += 1
    dom_key = max(per_k, key=lambda k: per_k[k]["ms"])
    dom = per_k[dom_key]
    model = dom["bytes"] / dom["n"]
    achieved = model / ((dom["ms"] / dom["n"]) * 1e-3) / 1e9
    cls = f"{dom_key[0]}|{KNAMES[dom_key[1]]}"
    traffic, prov = traffic_for(cls, model)
    roof = {"bound": "hbm", "kernel": cls, "achieved": round(achieved, 1), "peak": hbm,
            "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s", "frac": round(achieved / hbm, 4),
            "traffic": traffic,
            "traffic_unit": "DRAM bytes per call (dram__bytes_read.sum + dram__bytes_write.sum)",
            "traffic_source": prov,
            "algorithmic_bytes_per_call": int(model),
            "share_of_step": round(dom["ms"] / sum(v["ms"] for v in per_k.values()), 3),
            "note": "a call = feature pass + selector + the chosen kernel and its conversions, "
                    "one CUDA graph launch; CUDA events on the launch stream"}
    classes = {}
    for k, v in sorted(per_k.items(), key=lambda kv: -kv[1]["ms"]):
        t_call = v["ms"] / v["n"]
        classes[f"{k[0]}|{KNAMES[k[1]]}"] = {
            "calls": v["n"] // steps, "ms_per_step": round(v["ms"] / steps, 4), "us_per_call": round(t_call * 1e3, 1),
            "GBs": round(v["bytes"] / v["n"] / (t_call * 1e-3) / 1e9, 1),
            "frac": round(v["bytes"] / v["n"] / (t_call * 1e-3) / 1e9 / hbm, 4)}

    # end to end through the public API with pinned host buffers
    h2d, d2h = W.e2e_setup(torch)
    for _ in range(2):
        W.e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, steps // 2)
    e0.record()
    for _ in range(e2e_steps):
        W.e2e_step()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_val = step_bytes * world / (e2e_ms * 1e-3) / 1e9
    return {"value": round(value, 2), "ms_per_step": round(ms, 4), "step_work_bytes": int(step_bytes),
            "frac_of_hbm_roofline": round(value / world / hbm, 4), "roofline": roof,
            "e2e": {"value": round(e2e_val, 2), "unit": "GB/s", "ms_per_step": round(e2e_ms, 4),
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(steps * sum(c["launches"] for c in W.calls)),
            "clocks": clk, "wall_s_timed": round(wall, 3), "classes": classes}


def density_regret(W, torch, dev, reps=3):
    """Every forced candidate against the selector on each product of the
    stencil step (L2 flushed before every timing): the selected kernel, the
    fastest candidate, and regret = selector-driven time / fastest time."""
    hbm, _ = peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    for c in W.calls:
        times = {}
        for kk in ["auto"] + list(KNAMES):
            W.call(c, kk)
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                W.call(c, kk)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                if kk != "auto" and ts[-1] > 20 * times.get("auto", 1e9):
                    break  # far off the pace: one timing is enough
            times[kk] = float(np.median(ts))
        best = min(KNAMES, key=lambda q: times[q])
        rows.append({"call": c["kind"], "nnz_x": c["nnz_x"], "nnz_s": c["nnz_s"], "selected": KNAMES[c["kid"]],
                     "auto_us": round(times["auto"] * 1e3, 1), "best": best,
                     "best_us": round(times[best] * 1e3, 1), "regret": round(times["auto"] / times[best], 3),
                     "auto_GBs": round(c["bytes"] / (times["auto"] * 1e-3) / 1e9, 1),
                     "auto_frac": round(c["bytes"] / (times["auto"] * 1e-3) / 1e9 / hbm, 4),
                     "forced_us": {q: round(times[q] * 1e3, 1) for q in KNAMES}})
    return rows


def bench_batched(asv, torch, dev, reps=3):
    """4096 Zipf-row vectors through a 1M x 131072 lognormal/Zipf matrix: one
    batched call versus 4096 plain selector-driven calls into the same Y."""
    import gen
    m, n, B = 1_000_000, 131_072, 4096
    rp, c, v = gen.lognormal_zipf(m, n, np.log(40), 1.0, 1.2, gen.config_seed(3))
    # the vectors come from a second matrix over the same feature space (same popular columns)
    xrp_all, xc_all, xv_all = gen.lognormal_zipf(65_536, n, np.log(40), 1.0, 1.2, gen.config_seed(3) + 100,
                                                 perm_seed=gen.config_seed(3))
    pick = gen.randint(B, 65_536, gen.config_seed(3), 1)
    lens = (xrp_all[pick + 1] - xrp_all[pick]).astype(np.int64)
    xptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    xc = np.concatenate([xc_all[xrp_all[p]:xrp_all[p + 1]] for p in pick]).astype(np.int32)
    xv = np.concatenate([xv_all[xrp_all[p]:xrp_all[p + 1]] for p in pick]).astype(np.float32)
    A = asv.Matrix(m, n, torch.from_numpy(rp).to(dev), torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev))
    colptr_nnz = np.bincount(c, minlength=n)
    nnz_s = int(colptr_nnz[xc].sum())
    d_ptr, d_idx, d_val = (torch.from_numpy(a).to(dev) for a in (xptr, xc, xv))
    Y = torch.empty((B, m), dtype=torch.float32, device=dev)
    tune = A.autotune_batched(d_ptr, d_idx, d_val)
    A.spmspv_batched(d_ptr, d_idx, d_val, Y=Y)
    t_b = _time(torch, lambda: A.spmspv_batched(d_ptr, d_idx, d_val, Y=Y), reps)
    Yl = torch.empty_like(Y)
    cnts = [torch.tensor([int(lens[b])], dtype=torch.int64, device=dev) for b in range(B)]
    slices = [(d_idx[xptr[b]:xptr[b + 1]], d_val[xptr[b]:xptr[b + 1]]) for b in range(B)]

    def looped(kernel="auto"):
        for b in range(B):
            asv.asv_spmspv(A.handle, cnts[b], slices[b][0], slices[b][1], None, asv.ASV_OUT_DENSE, Yl[b],
                           kernel=kernel)
    # the same loop with each of the candidates that compete here forced, so
    # the batched form is also compared with the best fixed plain kernel
    fixed = {}
    for k in ("pull_warp", "push_warp_atom", "push_bal_atom"):
        looped(k)
        fixed[k] = round(_time(torch, lambda: looped(k), 1), 3)
    looped()
    t_l = _time(torch, looped, 1)
    diff = float(((Y - Yl).abs().max() / Yl.abs().max().clamp_min(1e-30)).item())
    ybytes = B * m * 4
    abytes = (m + 1) * 4 + len(c) * 8
    out = {"workload": "zipf 1M x 131072 (lognormal ln40/1.0, Zipf 1.2), 4096 vectors", "nnz": len(c),
           "entries": int(xptr[-1]), "multiply_adds": nnz_s, "tune": list(tune),
           "batched_ms": round(t_b, 3), "looped_ms": round(t_l, 3), "speedup_vs_looped": round(t_l / t_b, 2),
           "looped_fixed_ms": fixed, "speedup_vs_best_fixed_looped": round(min(fixed.values()) / t_b, 2),
           "looped_selector_regret": round(t_l / min(fixed.values()), 3),
           "batched_GBs": round((abytes + ybytes + xptr[-1] * 8) / (t_b * 1e-3) / 1e9, 1),
           "batched_Gmadds": round(nnz_s / (t_b * 1e-3) / 1e9, 1),
           "max_rel_diff_vs_looped": diff}
    del Y, Yl, A
    torch.cuda.empty_cache()
    return out


def bench_bfs(asv, torch, dev, W):
    """Whole breadth-first searches on the benchmark graph through the masked
    product (asv_bfs): the selector per level versus fixed candidates; GTEPS =
    edges of the reached component / time (Graph500 convention, each
    undirected edge counted once)."""
    import gen
    deg = np.diff(W.rowptr).astype(np.int64)
    out = {"workload": f"rmat scale {W.scale} edge factor {W.edge_factor}, {W.nroots} roots, Boolean handle"}
    level = torch.empty(W.n, dtype=torch.int32, device=dev)
    for k in ("auto", "pull_thread", "push_bal_atom", "mpull_bal"):
        W.Ab.bfs(W.roots[0], kernel=k, level=level)  # warm-up (graphs, workspaces)
        torch.cuda.synchronize()
        tot_ms, edges = 0.0, 0
        for r in W.roots:
            t0 = time.perf_counter()
            _, depth = W.Ab.bfs(r, kernel=k, level=level)
            torch.cuda.synchronize()
            tot_ms += (time.perf_counter() - t0) * 1e3
            lv = level.cpu().numpy()
            edges += int(deg[lv >= 0].sum()) // 2
        out[k] = {"ms_per_search": round(tot_ms / len(W.roots), 3), "GTEPS": round(edges / (tot_ms * 1e-3) / 1e9, 2)}
    # a high-diameter graph: the 5-point mesh 1024 x 1024 searched from a
    # corner (2047 levels, a thin frontier each), where per-level overheads rule
    side = 1024
    rp, c, _ = gen.laplace2d(side)
    nm = side * side
    M = asv.Matrix(nm, nm, torch.from_numpy(rp).to(dev), torch.from_numpy(c).to(dev), None)
    lv = torch.empty(nm, dtype=torch.int32, device=dev)
    mesh = {"workload": f"5-point mesh {side}x{side}, source at a corner, Boolean handle"}
    for k in ("auto", "push_warp_atom"):
        M.bfs(0, kernel=k, level=lv)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, depth = M.bfs(0, kernel=k, level=lv)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        mesh[k] = {"ms_per_search": round(ms, 2), "levels": depth, "us_per_level": round(ms * 1e3 / depth, 2)}
    out["mesh"] = mesh
    return out


def bench_pagerank(asv, torch, dev, W):
    """Incremental (delta-form) PageRank to a 1e-4 relative threshold on the
    benchmark graph through asv_pagerank: the selector per product versus a
    fixed pull and a fixed push candidate."""
    eps = 1e-4 * 0.15 / W.n
    out = {"workload": f"rmat scale {W.scale} edge factor {W.edge_factor}, damping 0.85, eps {eps:.3g}, FP32"}
    rank = torch.empty(W.n, dtype=torch.float32, device=dev)
    for k in ("auto", "pull_warp", "push_bal_atom"):
        W.Af.pagerank(0.85, eps, 100, kernel=k, rank=rank)  # warm-up (graphs, workspaces)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, iters = W.Af.pagerank(0.85, eps, 100, kernel=k, rank=rank)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        out[k] = {"ms": round(ms, 2), "products": iters, "ms_per_product": round(ms / max(iters, 1), 3)}
    return out


def bench_create(asv, torch, dev, W, reps=3):
    """Handle creation on the benchmark graph (once per matrix, outside the
    per-call cost): CSC view by radix sort, Table 1 features, merge-path
    partition, long-row segments. Bytes: CSR read (rowptr, col, values) plus
    the CSC written (colptr, rowidx, values, perm)."""
    out = {}
    for name, val in (("boolean", None), ("fp32", W.ones_d)):
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            A = asv.Matrix(W.m, W.n, W.rp_d, W.col_d, val)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            del A
        t = min(ts)
        sv = 0 if val is None else 4
        byt = 4 * (W.m + 1) + W.nnz * (4 + sv) + 4 * (W.n + 1) + W.nnz * (4 + sv + 4)
        out[name] = {"ms": round(t * 1e3, 2), "GBs_csr_to_csc": round(byt / t / 1e9, 1)}
    return out


def bench_backward(asv, torch, dev, reps=5):
    """16384^2 5%-dense layer, 64 activation vectors (5..50% dense): batched
    forward + fused backward versus 64 plain calls of each."""
    import gen
    m = n = 16384
    B = 64
    rp, c, v = gen.bernoulli(m, n, 0.05, 0.02, gen.config_seed(4))
    dens = gen.uniform(B, 0.05, 0.5, gen.config_seed(4), 1)
    X = gen.halfnormal(B * n, 1.0, gen.config_seed(4), 2).reshape(B, n)
    X = np.where(gen.uniform(B * n, 0, 1, gen.config_seed(4), 3).reshape(B, n) < dens[:, None], X, 0).astype(np.float32)
    dY = gen.uniform(B * m, -1, 1, gen.config_seed(4), 4, np.float32).reshape(B, m)
    A = asv.Matrix(m, n, torch.from_numpy(rp).to(dev), torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev))
    Xd, dYd = torch.from_numpy(X).to(dev), torch.from_numpy(dY).to(dev)
    Y = torch.empty((B, m), dtype=torch.float32, device=dev)
    dX = torch.empty((B, n), dtype=torch.float32, device=dev)
    dA = torch.empty(len(c), dtype=torch.float32, device=dev)
    A.autotune_batched(X_dense=Xd)
    t_fb = _time(torch, lambda: A.spmspv_batched(X_dense=Xd, Y=Y), reps)
    t_bb = _time(torch, lambda: asv.asv_spmspv_backward(A.handle, B, Xd, dYd, dX, dA), reps)
    Yl = torch.empty_like(Y)
    dXl = torch.empty_like(dX)
    dAl = torch.empty_like(dA)
    dA1 = torch.empty_like(dA)

    def fwd_loop():
        for b in range(B):
            asv.asv_spmspv(A.handle, None, None, None, Xd[b], asv.ASV_OUT_DENSE, Yl[b])

    def bwd_loop():
        dAl.zero_()
        for b in range(B):
            asv.asv_spmspv_backward(A.handle, 1, Xd[b], dYd[b], dXl[b], dA1)
            dAl.add_(dA1)
    fwd_loop()
    bwd_loop()
    t_fl = _time(torch, fwd_loop, 2)
    t_bl = _time(torch, bwd_loop, 2)
    rel = lambda a, b: float(((a - b).abs().max() / b.abs().max().clamp_min(1e-30)).item())
    out = {"workload": "16384^2 5% N(0,0.02) layer, 64 vectors 5-50% dense", "nnz": len(c),
           "forward_batched_ms": round(t_fb, 3), "forward_looped_ms": round(t_fl, 3),
           "forward_speedup": round(t_fl / t_fb, 2),
           "backward_fused_ms": round(t_bb, 3), "backward_looped_ms": round(t_bl, 3),
           "backward_speedup": round(t_bl / t_bb, 2),
           "max_rel_diff_vs_looped": {"y": rel(Y, Yl), "dx": rel(dX, dXl), "dA": rel(dA, dAl)}}
    del A
    torch.cuda.empty_cache()
    return out


def ncu_case(case, kernel, fmt="dense", density=None):
    """Small inputs (larger than L2, a few GB at most) for one-kernel profiles."""
    import torch

    import __graft_entry__ as ge
    import gen
    ge.build()
    import paper_2006_16767_gb300 as asv
    dev = torch.device("cuda")
    if case in ("stencil128", "rmat20"):
        if case == "stencil128":
            rp, c, v, _ = gen.stencil27(128, gen.config_seed(5))
            m = n = 128 ** 3
        else:
            rp, c = gen.rmat(20, 16, gen.config_seed(2))
            m = n = 1 << 20
            v = np.ones(len(c), np.float32)
        A = asv.Matrix(m, n, *[torch.from_numpy(a).to(dev) for a in (rp, c, v)])
        # --fmt dense: x dense, y dense; --fmt list: x as a list of every
        # column, y as the structural list (the two forms of the stencil step);
        # --density rho: x of round(rho n) random entries (list or dense) and,
        # with a list, a dense y (the stencil step's sparse-x calls)
        if density is None:
            idx = np.arange(n, dtype=np.int32)
            x = gen.uniform(n, -1, 1, 1, 0, np.float32)
        else:
            idx, xs = gen.sparse_x(n, max(1, int(round(density * n))), gen.config_seed(5), 11, np.float32)
            x = gen.densify(n, idx, xs, np.float32)
        xd = torch.from_numpy(x).to(dev)
        xl = torch.from_numpy(x[idx]).to(dev)
        it, cnt = torch.from_numpy(idx).to(dev), torch.tensor([n], dtype=torch.int64, device=dev)
        y = torch.empty(m, dtype=torch.float32, device=dev)
        yidx = torch.empty(m, dtype=torch.int32, device=dev)
        nnz_y = torch.zeros(1, dtype=torch.int64, device=dev)
        if density is not None:
            cnt = torch.tensor([len(idx)], dtype=torch.int64, device=dev)
        for _ in range(3):
            if fmt == "list" and density is not None:
                asv.asv_spmspv(A.handle, cnt, it, xl, None, asv.ASV_OUT_DENSE, y, kernel=kernel)
            elif fmt == "list":
                asv.asv_spmspv(A.handle, cnt, it, xl, None, asv.ASV_OUT_SPARSE, None, yidx, y, nnz_y, m, kernel)
            else:
                asv.asv_spmspv(A.handle, None, None, None, xd, asv.ASV_OUT_DENSE, y, kernel=kernel)
    elif case == "rmat20_bfs":
        # the densest BFS frontier of one root, Boolean, list in and list out (a BFS level product)
        rp, c = gen.rmat(20, 16, gen.config_seed(2))
        m = n = 1 << 20
        deg = np.diff(rp)
        root = int(np.flatnonzero(deg > 0)[0])
        fronts = bfs_frontiers(rp, c, [root])
        f = max(fronts, key=len)
        A = asv.Matrix(m, n, torch.from_numpy(rp).to(dev), torch.from_numpy(c).to(dev), None)
        fd = torch.from_numpy(f).to(dev)
        cnt = torch.tensor([len(f)], dtype=torch.int64, device=dev)
        yidx = torch.empty(m, dtype=torch.int32, device=dev)
        nnz_y = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(3):
            asv.asv_spmspv(A.handle, cnt, fd, None, None, asv.ASV_OUT_SPARSE, None, yidx, None, nnz_y, m, kernel)
        print("frontier", len(f), "of", n)
    elif case == "zipf_batched":
        m, n, B = 200_000, 131_072, 1024
        rp, c, v = gen.lognormal_zipf(m, n, np.log(40), 1.0, 1.2, gen.config_seed(3))
        xrp, xc, xv = gen.lognormal_zipf(B, n, np.log(40), 1.0, 1.2, gen.config_seed(3) + 100,
                                         perm_seed=gen.config_seed(3))
        A = asv.Matrix(m, n, *[torch.from_numpy(a).to(dev) for a in (rp, c, v)])
        args_ = [torch.from_numpy(a).to(dev) for a in (xrp.astype(np.int64), xc, xv)]
        # --kernel hot: the hot-column form (16 rows x 256 vectors, 64 hot columns)
        tune = (16, 256, 64) if kernel == "hot" else None
        for _ in range(3):
            A.spmspv_batched(*args_, tune=tune)
    elif case == "bernoulli_backward":
        m = n = 8192
        B = 64
        rp, c, v = gen.bernoulli(m, n, 0.05, 0.02, gen.config_seed(4))
        A = asv.Matrix(m, n, *[torch.from_numpy(a).to(dev) for a in (rp, c, v)])
        X = torch.from_numpy(gen.halfnormal(B * n, 1.0, 5).reshape(B, n)).to(dev)
        dY = torch.from_numpy(gen.uniform(B * m, -1, 1, 6, 0, np.float32).reshape(B, m)).to(dev)
        for _ in range(3):
            A.backward(X, dY)
    torch.cuda.synchronize()
    print("ok", case, kernel, fmt)


def density_sweep(which, out_path, reps=5):
    """Every candidate and the selector over x densities (x as a list with a
    dense y, and x dense with a dense y); L2 flushed before every timing."""
    import torch

    import __graft_entry__ as ge
    import gen
    ge.build()
    import paper_2006_16767_gb300 as asv
    dev = torch.device("cuda")
    if which == "stencil256":
        rp, c, v, _ = gen.stencil27(256, gen.config_seed(5))
        m = n = 256 ** 3
        rhos = [1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0]
    else:
        rp, c = gen.rmat(22, 16, gen.config_seed(2))
        m = n = 1 << 22
        v = np.ones(len(c), np.float32)
        rhos = [1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 0.3, 1.0]
    nnz = len(c)
    colcount = np.bincount(c, minlength=n)
    A = asv.Matrix(m, n, *[torch.from_numpy(a).to(dev) for a in (rp, c, v)])
    y = torch.empty(m, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    hbm, _ = peaks()
    out = open(out_path, "w")
    for rho in rhos:
        k = max(1, int(round(rho * n)))
        idx, val = gen.sparse_x(n, k, gen.config_seed(5), 11, np.float32)
        it, vt = torch.from_numpy(idx).to(dev), torch.from_numpy(val).to(dev)
        cnt = torch.tensor([len(idx)], dtype=torch.int64, device=dev)
        xd = torch.zeros(n, dtype=torch.float32, device=dev)
        xd[it.long()] = vt
        nnz_s = int(colcount[idx].sum())
        for fmt, dense_x in (("list_x", False), ("dense_x", True)):
            def call(kk):
                asv.asv_spmspv(A.handle, cnt, it, vt, xd if dense_x else None, asv.ASV_OUT_DENSE, y, kernel=kk)
            times = {}
            for kk in ["auto"] + list(asv.KERNELS):
                call(kk)
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    call(kk)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                    if ts[-1] > 50 * min(times.values(), default=1e9):
                        break
                times[kk] = float(np.median(ts))
            kid, _ = asv.asv_select(A.handle, cnt, it, vt, xd if dense_x else None)
            best_k = min(asv.KERNELS, key=lambda q: times[q])
            work = work_bytes(m, n, nnz, k, nnz_s, m, 4, 4, 4, not dense_x, False)
            rec = {"matrix": which, "format": fmt, "rho": rho, "nnz_x": k, "nnz_s": nnz_s,
                   "selected": asv.KERNELS[kid], "auto_ms": round(times["auto"], 4),
                   "best": best_k, "best_ms": round(times[best_k], 4),
                   "regret": round(times["auto"] / times[best_k], 3),
                   "auto_GBs": round(work / (times["auto"] * 1e-3) / 1e9, 1),
                   "auto_frac": round(work / (times["auto"] * 1e-3) / 1e9 / hbm, 4),
                   "auto_GFLOPs": round(2 * nnz_s / (times["auto"] * 1e-3) / 1e9, 2),
                   "ms": {q: round(times[q], 4) for q in asv.KERNELS}}
            out.write(json.dumps(rec) + "\n")
            out.flush()
            print(json.dumps({k2: rec[k2] for k2 in ("matrix", "format", "rho", "selected", "auto_ms", "best",
                                                     "best_ms", "regret", "auto_frac")}), flush=True)
    out.close()


def cpu_baseline(W):
    """The oracle on the host cores: its multi-threaded form on every core
    (the line's figure) and its serial form on one."""
    import oracle
    out = {"kind": "oracle", "unit": "GB/s"}
    try:
        threads = oracle.par_threads()
        W.oracle_step(par=True)  # warm (page-in, thread pool)
        b, t = W.oracle_step(par=True)
        out.update({"value": round(b / t / 1e9, 4), "cores": threads, "seconds": round(t, 3),
                    "sample": f"one whole step of {W.name} ({len(W.calls)} products), multi-threaded FP64 C oracle "
                              f"(row-parallel pull, column-parallel push) on {threads} threads"})
    except (OSError, subprocess.CalledProcessError) as e:
        out["parallel_unavailable"] = str(e)[:200]
    b, t = W.oracle_step(par=False)
    serial = {"value": round(b / t / 1e9, 4), "cores": 1, "seconds": round(t, 3),
              "sample": f"one whole step of {W.name}, serial FP64 C oracle"}
    if "value" not in out:
        out.update(serial)
    else:
        out["serial"] = serial
    return out


# ------------------------------------------------------------------ main
def make_workload(name):
    if name in ("stencil256", Stencil256.name):
        return Stencil256()
    if name in ("rmat22", Rmat22.name):
        return Rmat22()
    raise SystemExit(f"unknown workload {name}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stencil256", help="stencil256 (default) or rmat22")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip every section but the headline step")
    ap.add_argument("--ncu-case", default=None,
                    help="profiling aid: run one small case (stencil128, rmat20, rmat20_bfs, zipf_batched, "
                         "bernoulli_backward) with --kernel (and --fmt) three times and exit")
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--fmt", default="dense", choices=["dense", "list"])
    ap.add_argument("--density", type=float, default=None,
                    help="with --ncu-case stencil128: x of this density instead of a full one")
    ap.add_argument("--sweep", default=None,
                    help="x-density sweep of every candidate and the selector on stencil256 or rmat22; "
                         "writes JSON lines to --sweep-out")
    ap.add_argument("--sweep-out", default="sweep.jsonl")
    ap.add_argument("--direct", action="store_true",
                    help="profiling aid: run the recorded kernel choices as direct launches instead of the "
                         "selector graph (the profiler cannot see kernels inside conditional graph nodes)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return main_reference(args, rank, world)
    if args.ncu_case:
        return ncu_case(args.ncu_case, args.kernel, args.fmt, args.density)
    if args.sweep:
        return density_sweep(args.sweep, args.sweep_out)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    import paper_2006_16767_gb300 as asv

    W = make_workload(args.workload)
    W.setup_gpu(asv, torch, dev)
    res = measure(W, torch, dev, args.steps, args.warmup, direct=args.direct, world=world, dist=dist,
                  clocks_index=local)
    out = {"metric": METRIC, "value": res["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": res["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": W.dtype, "data": "synthetic", "config": W.config(),
           "frac_of_hbm_roofline": res["frac_of_hbm_roofline"], "roofline": res["roofline"], "e2e": res["e2e"],
           "gpu_launches": res["gpu_launches"], "clocks": res["clocks"], "wall_s_timed": res["wall_s_timed"],
           "step_work_bytes": res["step_work_bytes"], "classes": res["classes"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(W)
    if not args.no_extra:
        if isinstance(W, Stencil256):
            out["density_regret"] = density_regret(W, torch, dev)
            del W
            torch.cuda.empty_cache()
            R = Rmat22()
            R.setup_gpu(asv, torch, dev)
            r = measure(R, torch, dev, max(3, args.steps // 2), args.warmup)
            r.pop("clocks", None)
            out["rmat22"] = dict(config=R.config(), **r)
        else:
            R = W
        out["bfs"] = bench_bfs(asv, torch, dev, R)
        out["create"] = bench_create(asv, torch, dev, R)
        out["pagerank_incremental"] = bench_pagerank(asv, torch, dev, R)
        del R
        torch.cuda.empty_cache()
        out["batched"] = bench_batched(asv, torch, dev)
        out["backward"] = bench_backward(asv, torch, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def main_reference(args, rank, world):
    """The oracle (CPU; its multi-threaded form on every host core) on the
    same workload, metric and unit; rank 0 only."""
    if rank != 0:
        return
    import oracle
    W = make_workload(args.workload)
    if isinstance(W, Stencil256):
        W.plan_calls_host()
    else:
        fronts = []
        for r in W.roots:
            fronts += oracle.frontiers(W.n, W.rowptr, W.col, r)
        W.frontiers_host = fronts
        colptr, _, _ = oracle.csr_to_csc(W.m, W.n, W.rowptr, W.col)
        W.calls = []
        for f in fronts:
            vf = oracle.vector_features(W.n, W.nnz, colptr, f)
            xb = np.zeros(W.n, np.uint8)
            xb[f] = 1
            nnz_y = int(oracle.bool_pull(W.rowptr, W.col, xb).sum())
            W.calls.append(dict(kind="bfs", nnz_x=len(f), nnz_s=vf["nnz_s"],
                                bytes=work_bytes(W.m, W.n, W.nnz, len(f), vf["nnz_s"], nnz_y, 0, 0, 0, True, True)))
        W.calls.append(dict(kind="pagerank", nnz_x=W.n, nnz_s=W.nnz,
                            bytes=work_bytes(W.m, W.n, W.nnz, W.n, W.nnz, W.m, 4, 4, 4, False, False)))
    try:
        par, threads = True, oracle.par_threads()
    except (OSError, subprocess.CalledProcessError):
        par, threads = False, 1
    for _ in range(args.warmup):
        W.oracle_step(par=par)
    tot_b, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        b, t = W.oracle_step(par=par)
        tot_b += b
        tot_t += t
    ms = tot_t / args.steps * 1e3
    val = tot_b / tot_t / 1e9
    form = f"multi-threaded FP64 C oracle on {threads} threads" if par else "serial FP64 C oracle"
    out = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle)", "data": "synthetic",
           "config": W.config(),
           "cpu_baseline": {"kind": "oracle", "cores": threads, "value": round(val, 4), "unit": "GB/s",
                            "sample": f"per step: one whole step of {W.name} ({len(W.calls)} products), {form}"},
           "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
