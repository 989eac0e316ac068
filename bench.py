"""Benchmark: the site-local lattice-expression hot path on one GB300 per rank.

One step = one pass of every hot-path row over synthetic inputs of the 48^4
volume-sweep configuration (5,308,416 sites):
  A2 z=a*b (FP64 storage), A3 z=a*v, A4 Lorentz z_mu=a_mu*b_mu (mu=0..3),
  A5 fused z=a*b+c*d, z=a*b*c+0.5*d, z=adj(a)*b-b*adj(a),
  A6 z=a*b stored in FP32 / BF16 / FP16 (FP32 accumulation),
  A7 z=a*b in two-row (12-real) SU(3) storage, FP64 and FP32,
  A8 64 lattices of mixed volumes, z=a*b+c*d each, one CUDA-graph launch,
  A9 reverse mode of z=a*b and of z=a*b+c*d.
Before timing, the library's autotuner picks each row's launch shape and data
movement (setup, outside the timed region; --no-tune keeps the defaults).
`value` is the aggregate algorithmic bandwidth of the step (STREAM
convention: every input read once, every output written once) with inputs
resident in HBM; every field is larger than the 129 MB L2, so no flush is
needed between steps.  `e2e` runs the same step through the C ABI from pinned
host buffers that hold each field in its storage format (upload + layout
kernel, evaluate, layout kernel + download inside the timed region).
`--impl reference` times the CPU oracle on a bounded sample, on every host core
(one spawned process per core, each on its own sites).  The studies
(`--study`) measure beside the step; the errors against the oracle are
measured by the GPU tests (tests/test_gpu_error_study.py), not here.

Multi-GPU (torchrun): every rank runs its own copy of the step (independent
lattices, no collective on the data path); value = total bytes of all ranks /
max time over ranks (weak scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("SU(3)xSU(3) stream GB/s & sites/s, % HBM peak; FP64 vs reduced-prec at stated error")
DIMS = (48, 48, 48, 48)
SEED = 1710094090 + 1
BATCH_SHAPES = [(4, 4, 4, 4), (8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 24)]

# algorithmic bytes per site (inputs read once, outputs written once)
B_MM, B_MV, B_E1, B_E2, B_E3 = 432, 240, 720, 720, 432
B_F32, B_H, B_C12, B_C12F = 216, 108, 288, 144
B_ADJ_MM, B_ADJ_E1 = 720, 1296
ROW_NAMES = ["A2 z=a*b", "A3 z=a*v", "A4 z_mu=a_mu*b_mu", "A5 z=a*b+c*d", "A5 z=a*b*c+0.5*d",
             "A5 z=adj(a)*b-b*adj(a)", "A6 z=a*b f32", "A6 z=a*b bf16", "A6 z=a*b f16",
             "A7 z=a*b f64_c12", "A7 z=a*b f32_c12", "A8 batch 64 lattices z=a*b+c*d",
             "A9 adjoint of z=a*b", "A9 adjoint of z=a*b+c*d"]
ROW_A8, ROW_A9A, ROW_A9B = ROW_NAMES[11], ROW_NAMES[12], ROW_NAMES[13]
MATH_NAMES = ("fx", "df32", "f64")
MATH_IDS = {"f64": 1, "df32": 2, "fx": 3}
MATH_DESC = {"fx": "shared-exponent fixed-point (fx)", "df32": "pair-of-FP32 (df32)",
             "f64": "native FP64 (f64)"}
# arithmetic type of the rows with FP64 storage under each arithmetic
MATH_DTYPE = {"fx": "int64", "df32": "df32", "f64": "f64"}
# maximum absolute error against the FP64 oracle over every output, from the
# error tests (tests/test_gpu_error_study.py): df32 over every output of every
# FP64-storage row of the 48^4 step (SU(3) operands; the Gaussian-operand rows
# A3 and A9 reach 1.3e-13 - 1.6e-13, within the bound scaled by the operands'
# size); fx and f64 over the fused trees at 32^4 and a*b at 48^4
MATH_ERR = {"fx": "7.8e-16 - 1.6e-15",
            "df32": "3.9e-14 - 6.0e-14 (SU(3) operands, every output of the 48^4 step)",
            "f64": "3.3e-16 - 6.7e-16"}

# The tree each FP64-storage row evaluates (pair arithmetic), as the kernels'
# template arguments name it: (tree, arithmetic type, storage, reverse mode).
# With the data movement the row ran with (the tuner's variant, else the
# library's default) this gives the kernel ncu names; the reverse mode of
# a*b+c*d runs split (two launches of the single-product reverse kernel) when
# the tuner chose that (reported variant 10 + the halves' variant).
T_MM = "Mul<LM<0>, LM<1>>"
T_E1 = "Add<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>"
ROW_TREE = {
    "A2 z=a*b": (T_MM, "MathDF", 0, False),
    "A3 z=a*v": ("Mul<LM<0>, LV<1>>", "MathDF", 0, False),
    "A4 z_mu=a_mu*b_mu": (T_MM, "MathDF", 0, False),
    "A5 z=a*b+c*d": (T_E1, "MathDF", 0, False),
    "A5 z=a*b*c+0.5*d": ("Add<Mul<Mul<LM<0>, LM<1>>, LM<2>>, Scale<0, LM<3>>>", "MathDF", 0, False),
    "A5 z=adj(a)*b-b*adj(a)": ("Sub<Mul<Adj<LM<0>>, LM<1>>, Mul<LM<1>, Adj<LM<0>>>>", "MathDF", 0, False),
    "A7 z=a*b f64_c12": (T_MM, "MathDF", 4, False),
    "A9 adjoint of z=a*b": (T_MM, "MathDF", 0, True),
    "A9 adjoint of z=a*b+c*d": (T_E1, "MathDFScalar", 0, True),
}
ROW_KERNEL_FIXED = {
    "A8 batch 64 lattices z=a*b+c*d": "k_batch_tma<MathDF, Add<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>>",
}
FWD_KERNEL = ["k_eval<{t}, {m}, {p}>", "k_eval_tma<{t}, {m}, {p}>", "k_eval_lazy<{t}, {m}, {p}>",
              "k_eval_ring<{t}, {m}, {p}>", "k_eval_pair<{t}>"]
ADJ_KERNEL = ["k_adjoint<{t}, {m}>", "k_adjoint_tma<{t}, {m}>", "k_adjoint_lazy<{t}, {m}>",
              "k_adjoint_ring<{t}, {m}>", "k_adjoint_pair<{t}>"]
# the library's default data movement of each row's kernel when untuned
ROW_DEFAULT_VARIANT = {"A9 adjoint of z=a*b": 4, "A9 adjoint of z=a*b+c*d": 14}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel on a 32^4 lattice (1,048,576 sites; the batch row: its 64 fixed
# lattices), from one ncu capture of that kernel in the benchmark's rows as
# they stand (default launches, one launch after the warm-up): (bytes,
# algorithmic bytes of that launch); scaled to the benchmark's volume in
# proportion to the algorithmic bytes.  A kernel missing here reports traffic
# null.
TRAFFIC_32 = {
    "k_eval_tma<Mul<LM<0>, LM<1>>, MathDF, 0>": (414.5 * 1e6, 452984832),
    "k_eval_tma<Mul<LM<0>, LV<1>>, MathDF, 0>": (228.6 * 1e6, 251658240),
    "k_eval_tma<Add<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>, MathDF, 0>": (729.2 * 1e6, 754974720),
    "k_eval_tma<Add<Mul<Mul<LM<0>, LM<1>>, LM<2>>, Scale<0, LM<3>>>, MathDF, 0>": (728.5 * 1e6, 754974720),
    "k_eval_tma<Sub<Mul<Adj<LM<0>>, LM<1>>, Mul<LM<1>, Adj<LM<0>>>>, MathDF, 0>": (414.7 * 1e6, 452984832),
    "k_eval_tma<Mul<LM<0>, LM<1>>, MathDF, 4>": (265.2 * 1e6, 301989888),
    "k_batch_tma<MathDF, Add<Mul<LM<0>, LM<1>>, Mul<LM<2>, LM<3>>>>": (4602.2 * 1e6, 4622376960),
    "k_adjoint_tma<Mul<LM<0>, LM<1>>, MathDF>": (703.6 * 1e6, 754974720),
    "k_adjoint_pair<Mul<LM<0>, LM<1>>>": (701.6 * 1e6, 754974720),
}


def traffic_bytes(kernel, nbytes):
    """Measured DRAM bytes of one launch of a kernel, scaled to nbytes."""
    t = TRAFFIC_32.get(kernel)
    if t is None:
        return None
    return int(round(t[0] * nbytes / t[1]))


def row_launches(r, tuned_variant):
    """(kernel, launches, algorithmic bytes per launch) of a row as it ran."""
    if r.name in ROW_KERNEL_FIXED:
        return ROW_KERNEL_FIXED[r.name], 1, r.nbytes
    if r.name not in ROW_TREE:
        return r.name, 1, r.nbytes
    tree, math, prec, adj = ROW_TREE[r.name]
    v = tuned_variant if tuned_variant is not None else ROW_DEFAULT_VARIANT.get(r.name, 1)
    if adj and v >= 10:
        return ADJ_KERNEL[v - 10].format(t=T_MM, m="MathDF"), 2, B_ADJ_MM * r.sites
    names = ADJ_KERNEL if adj else FWD_KERNEL
    return names[v].format(t=tree, m=math, p=prec), 1, r.nbytes


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """Maximum of a per-rank scalar over all ranks (identity without a group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_rank_step, ws, ms_per_step_max):
    """Whole-job bandwidth: bytes of all ranks over the slowest rank's time."""
    return bytes_per_rank_step * ws / (ms_per_step_max * 1e-3) / 1e9


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows),
                "power_w_max": max([float(r[2]) for r in self.rows
                                    if r[2].replace(".", "").isdigit()] or [0.0])}


# ------------------------------------------------------------------ rows
class Row:
    def __init__(self, name, nbytes, sites, run, inputs, outputs, launches=1, dtype="f64"):
        self.name, self.nbytes, self.sites, self.run = name, nbytes, sites, run
        self.inputs, self.outputs, self.launches, self.dtype = inputs, outputs, launches, dtype
        self.ms = []
        self.tune = None   # callable(stream) -> (threads, blocks/SM, variant, ms), forward rows


def out_buf_bytes(dims):
    """Largest output of the step: the Lorentz product, 4 FP64 matrices per site."""
    v = 1
    for x in dims:
        v *= x
    return 4 * 144 * v


def e2e_host_bytes(dims):
    """Pinned host memory one rank's end-to-end run holds: the canonical FP64
    inputs (a, b, c, d, W: 144 B per site each; v 48; the two Lorentz fields
    576 each), the stored copies of the reduced-precision and two-row inputs
    (576 B per site in all), the 64 batch lattices (4 FP64 matrix fields over
    their 6.2 M sites) and two output buffers of the largest output."""
    v = 1
    for x in dims:
        v *= x
    batch = 4 * 144 * sum(int(np.prod(s)) * 13 for s in BATCH_SHAPES)   # ~64 lattices
    return (5 * 144 + 48 + 2 * 576 + 576) * v + batch + 2 * out_buf_bytes(dims)


def host_mem_available():
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def e2e_host_shortage(dims, local_ranks, available):
    """None if every rank on this node can pin its end-to-end buffers (at most
    85% of the available host memory in all), else the reason, one line."""
    need = e2e_host_bytes(dims) * local_ranks
    if available is None or need <= 0.85 * available:
        return None
    return ("host memory: %d ranks need %.0f GB pinned, %.0f GB available"
            % (local_ranks, need / 1e9, available / 1e9))


def build_rows(su3s, synth, torch, with_host, dims=DIMS, want=lambda name: True):
    """Allocate fields, fill them from the seeded generator, return the rows
    whose names pass `want`."""
    v = synth.volume(dims)
    lat = su3s.Lattice(dims)
    F64, MATRIX, VECTOR = su3s.F64, su3s.MATRIX, su3s.VECTOR
    host = {}

    def gen(kind, field, n, nmu=1, dims=None, seed=SEED):
        if kind == "su3":
            arr = synth.su3(seed, field, n * nmu)
        elif kind == "gm":
            arr = synth.gauss_matrix(seed, field, n * nmu)
        else:
            arr = synth.gauss_vector(seed, field, n * nmu)
        return arr

    def pinned(arr):
        t = torch.from_numpy(arr.reshape(-1))
        return t.pin_memory() if with_host else None

    def field(lat_, kind, nmu, prec, arr):
        f = su3s.Field(lat_, kind, nmu, prec, su3s.SOA)
        f.upload(arr)
        return f

    H = {}
    need = {"a": any(want(n) for n in ROW_NAMES if "A8" not in n),
            "b": any(want(n) for n in ROW_NAMES if "A8" not in n),
            "c": any(want(n) for n in ROW_NAMES if ("c*d" in n or "*c" in n) and "A8" not in n),
            "v": want("A3 z=a*v"), "w": any(want(n) for n in ROW_NAMES if "A9" in n),
            "l": want("A4 z_mu=a_mu*b_mu")}
    for n, fid in (("a", 0), ("b", 1), ("c", 2), ("d", 3)):
        if need["c" if n in "cd" else n]:
            H[n] = gen("su3", fid, v)
    if need["v"]:
        H["v"] = gen("vec", 4, v)
    if need["w"]:
        H["w"] = gen("gm", 5, v)
    if need["l"]:
        H["la"] = gen("su3", 0, v, 4)
        H["lb"] = gen("su3", 1, v, 4)
    P = {k: pinned(a) for k, a in H.items()}

    def fields_for(prec, names=("a", "b", "c", "d")):
        return {n: field(lat, MATRIX, 1, prec, H[n]) for n in names if n in H}

    Fd = fields_for(F64)
    Fv = field(lat, VECTOR, 1, F64, H["v"]) if "v" in H else None
    Fw = field(lat, MATRIX, 1, F64, H["w"]) if "w" in H else None
    La = field(lat, MATRIX, 4, F64, H["la"]) if "la" in H else None
    Lb = field(lat, MATRIX, 4, F64, H["lb"]) if "lb" in H else None
    rows = []

    shared_out = {}

    def out_pin(f):
        # every output is downloaded into one of two pinned byte buffers (one
        # per download stream: downloads on one stream are ordered, so they
        # never overlap), viewed with the output's stored shape and dtype
        if not with_host:
            return None
        nb = int(np.prod(f.stored_shape)) * torch.empty(0, dtype=f.stored_dtype).element_size()
        if not shared_out or shared_out["bytes"] < nb:
            cap = max(nb, out_buf_bytes(dims))
            shared_out.update(bytes=cap, bufs=[torch.empty(cap, dtype=torch.uint8).pin_memory()
                                               for _ in range(2)])
        return tuple(b[:nb].view(f.stored_dtype).view(f.stored_shape) for b in shared_out["bufs"])

    def mk(name, bps, dest, expr, ins, dtype="f64"):
        def run(stream, dest=dest, expr=expr):
            su3s.evaluate(dest, expr, su3s.MATH_DEFAULT, stream)
            return 1
        r = Row(name, bps * v * dest.nmu, v * dest.nmu, run, ins, [(dest, out_pin(dest))],
                dtype=dtype)
        r.tune = lambda stream, dest=dest, expr=expr: su3s.tune(dest, expr, su3s.MATH_DEFAULT,
                                                                 stream)
        return r

    if want("A2 z=a*b"):
        z = Fd["a"].like()
        rows.append(mk("A2 z=a*b", B_MM, z, Fd["a"] * Fd["b"],
                       [(Fd["a"], P["a"]), (Fd["b"], P["b"])]))
    if want("A3 z=a*v"):
        zv = Fv.like()
        rows.append(mk("A3 z=a*v", B_MV, zv, Fd["a"] * Fv, [(Fd["a"], P["a"]), (Fv, P["v"])]))
    if want("A4 z_mu=a_mu*b_mu"):
        zl = La.like()
        rows.append(mk("A4 z_mu=a_mu*b_mu", B_MM, zl, La * Lb, [(La, P["la"]), (Lb, P["lb"])]))
    if "a" in Fd:
        a, b = Fd["a"], Fd["b"]
    if "c" in Fd:
        c, d = Fd["c"], Fd["d"]
    if want("A5 z=a*b+c*d"):
        rows.append(mk("A5 z=a*b+c*d", B_E1, a.like(), a * b + c * d,
                       [(Fd[n], P[n]) for n in "abcd"]))
    if want("A5 z=a*b*c+0.5*d"):
        rows.append(mk("A5 z=a*b*c+0.5*d", B_E2, a.like(), a * b * c + 0.5 * d,
                       [(Fd[n], P[n]) for n in "abcd"]))
    if want("A5 z=adj(a)*b-b*adj(a)"):
        rows.append(mk("A5 z=adj(a)*b-b*adj(a)", B_E3, a.like(), a.adj() * b - b * a.adj(),
                       [(Fd[n], P[n]) for n in "ab"]))
    for prec, nm, bps in ((su3s.F32, "f32", B_F32), (su3s.BF16, "bf16", B_H), (su3s.F16, "f16", B_H),
                          (su3s.F64_C12, "f64_c12", B_C12), (su3s.F32_C12, "f32_c12", B_C12F)):
        tag = "A7" if "c12" in nm else "A6"
        name = "%s z=a*b %s" % (tag, nm)
        if not want(name):
            continue
        Fp = fields_for(prec, ("a", "b"))
        zp = Fp["a"].like()
        rows.append(mk(name, bps, zp, Fp["a"] * Fp["b"],
                       [(Fp["a"], P["a"]), (Fp["b"], P["b"])], dtype=nm))

    # A8: 64 lattices of mixed volumes, one graph launch
    if not want(ROW_A8):
        return _adjoint_rows(su3s, rows, want, v, Fd, Fw, P, out_pin), {"lat": lat}
    picks = (synth.uniform_real(SEED + 3, 40, 64) + 1.0) / 2.0 * len(BATCH_SHAPES)
    batch = su3s.Batch()
    bins, bouts, bsites = [], [], 0
    keep = []
    for i, p in enumerate(picks):
        bdims = BATCH_SHAPES[min(int(p), len(BATCH_SHAPES) - 1)]
        bl = su3s.Lattice(bdims)
        nv = synth.volume(bdims)
        fs = {}
        for n in "abcd":
            arr = synth.su3(SEED + 3 + 1000 * i, synth.FIELD[n], nv)
            fs[n] = field(bl, MATRIX, 1, F64, arr)
            bins.append((fs[n], pinned(arr)))
        zb = fs["a"].like()
        batch.add(zb, fs["a"] * fs["b"] + fs["c"] * fs["d"])
        bouts.append((zb, out_pin(zb)))
        bsites += nv
        keep.append((bl, fs, zb))
    batch.build()

    def run_batch(stream):
        batch.launch(stream)
        return 1
    rows.append(Row(ROW_A8, B_E1 * bsites, bsites, run_batch, bins, bouts))
    rows[-1].keep = (batch, keep)

    def tune_batch(stream):
        th, tile, bps, ms = batch.tune(su3s.MATH_DEFAULT, stream)
        return {"threads": th, "blocks_per_sm": bps, "tile_sites": tile, "ms": round(ms, 5)}
    rows[-1].tune = tune_batch

    return _adjoint_rows(su3s, rows, want, v, Fd, Fw, P, out_pin), {"lat": lat}


def _adjoint_rows(su3s, rows, want, v, Fd, Fw, P, out_pin):
    """A9: reverse mode of z=a*b and of z=a*b+c*d."""
    if want(ROW_A9A):
        a, b = Fd["a"], Fd["b"]
        ga, gb = a.like(), a.like()

        def run_adj(stream):
            su3s.eval_adjoint(a * b, Fw, [ga, gb], su3s.MATH_DEFAULT, stream)
            return 1
        rows.append(Row(ROW_A9A, B_ADJ_MM * v, v, run_adj,
                        [(a, P["a"]), (b, P["b"]), (Fw, P["w"])],
                        [(ga, out_pin(ga)), (gb, out_pin(gb))]))
        rows[-1].tune = lambda stream, a=a, b=b, ga=ga, gb=gb: su3s.tune_adjoint(
            a * b, Fw, [ga, gb], su3s.MATH_DEFAULT, stream)
    if want(ROW_A9B):
        a, b, c, d = (Fd[n] for n in "abcd")
        g4 = [a.like() for _ in range(4)]
        e1 = a * b + c * d

        def run_adj1(stream):
            su3s.eval_adjoint(e1, Fw, g4, su3s.MATH_DEFAULT, stream)
            return 1
        rows.append(Row(ROW_A9B, B_ADJ_E1 * v, v, run_adj1,
                        [(Fd[n], P[n]) for n in "abcd"] + [(Fw, P["w"])],
                        [(g, out_pin(g)) for g in g4]))
        rows[-1].tune = lambda stream, e1=e1, g4=g4: su3s.tune_adjoint(
            e1, Fw, g4, su3s.MATH_DEFAULT, stream)
    return rows


def time_step(rows, torch, stream, steps, warmup, per_row_events=True):
    """Run `steps` steps; return (total ms from the outer events, per-row ms lists)."""
    for _ in range(warmup):
        for r in rows:
            r.run(stream)
    stream.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in rows] for _ in range(steps)] if per_row_events else None
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    start.record(stream)
    for k in range(steps):
        for i, r in enumerate(rows):
            if ev:
                ev[k][i][0].record(stream)
            launches += r.run(stream)
            if ev:
                ev[k][i][1].record(stream)
    end.record(stream)
    end.synchronize()
    total = start.elapsed_time(end)
    per_row = [[ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(steps)] for i in range(len(rows))] \
        if ev else None
    return total, per_row, launches


def stored_host(f, canon, torch):
    """The pinned host array a user holding field `f` in its storage format
    has: for FP64 fields the canonical array itself; for reduced precisions the
    values converted by torch on the host; for two-row formats rows 0 and 1
    only."""
    if f.prec == 0 or f.kind == 2:
        return canon.view(f.stored_shape)
    x = canon.view((-1,) + tuple(f.canonical_shape[1:]))
    if f.stored_shape[1] == 6:
        x = x[:, :2].reshape(-1, 6, 2)
    return x.reshape(f.stored_shape).to(f.stored_dtype).contiguous().pin_memory()


def time_e2e(rows, torch, stream, steps):
    """The step through the C ABI from pinned host buffers, each field held on
    the host in its storage format.  Every distinct input field is uploaded
    (H2D copy + layout kernel) once per step on one of
    two upload streams, each row runs on the compute stream as soon as its
    inputs are in, and its outputs are unpacked and copied back on one of two
    download streams; events order them, so host->device copies, kernels and
    device->host copies of different rows (and of consecutive steps) overlap: a
    field is overwritten only after the previous step's download of it, and a
    copy does not wait for the previous field's layout kernel.  Returns (ms per step, H2D
    bytes, D2H bytes)."""
    ups = [torch.cuda.Stream(), torch.cuda.Stream()]
    downs = [torch.cuda.Stream(), torch.cuda.Stream()]
    comp = stream
    fields, order = {}, []
    for r in rows:
        for f, h in r.inputs:
            if id(f) not in fields:
                fields[id(f)] = (f, stored_host(f, h, torch))
                order.append(id(f))
    last_use, fetched = {}, {}

    def one():
        ready = {}
        for k, fid in enumerate(order):
            f, h = fields[fid]
            up = ups[k % 2]
            if fid in last_use:                 # previous step's readers are done with f
                up.wait_event(last_use[fid])
            f.upload_stored(h, up)
            ev = torch.cuda.Event()
            ev.record(up)
            ready[fid] = ev
        nout = 0
        for r in rows:
            for f, _ in r.inputs:
                comp.wait_event(ready[id(f)])
            for f, _ in r.outputs:              # previous step's download of f is done
                if id(f) in fetched:
                    comp.wait_event(fetched[id(f)])
            r.run(comp)
            done = torch.cuda.Event()
            done.record(comp)
            for f, _ in r.inputs:
                last_use[id(f)] = done
            for f, h in r.outputs:
                down, buf = downs[nout % 2], h[nout % 2]
                nout += 1
                down.wait_event(done)
                f.download_stored(out=buf, stream=down)
                ev = torch.cuda.Event()
                ev.record(down)
                fetched[id(f)] = ev

    one()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(comp)
    for st_ in ups + downs:
        st_.wait_stream(comp)
    for _ in range(steps):
        one()
    for down in downs:                          # the last step's downloads are in
        comp.wait_stream(down)
    end.record(comp)
    end.synchronize()
    torch.cuda.synchronize()
    h2d = sum(fields[fid][1].numel() * fields[fid][1].element_size() for fid in order)
    d2h = sum(h[0].numel() * h[0].element_size() for r in rows for _, h in r.outputs)
    return start.elapsed_time(end) / steps, h2d, d2h


def measure_link(torch, nbytes=1 << 30, reps=3):
    """Host link bandwidth as the e2e step uses it: one pinned host->device and
    one device->host copy of nbytes each, concurrently on two streams; best of
    reps, in GB/s of both directions together."""
    hs = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hd = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    ds = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dd = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = 0.0
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s1)
        s2.wait_event(t0)
        with torch.cuda.stream(s1):
            ds.copy_(hs, non_blocking=True)
        with torch.cuda.stream(s2):
            hd.copy_(dd, non_blocking=True)
        s1.wait_stream(s2)
        t1.record(s1)
        t1.synchronize()
        best = max(best, 2 * nbytes / (t0.elapsed_time(t1) * 1e-3) / 1e9)
    del hs, hd, ds, dd
    return best


# ----------------------------------------------------------- CPU oracle
def _oracle_pass_worker(job):
    """One worker of the CPU baseline: the oracle, as it stands (single-threaded
    C), on `n` sites starting at `first`: every row's computation, repeated
    until `budget_s` has passed.  Runs in a spawned process."""
    first, n, budget_s = job
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    a, b, c, d = (synth.su3(SEED, i, n, first=first) for i in range(4))
    vv = synth.gauss_vector(SEED, 4, n, first=first)
    w = synth.gauss_matrix(SEED, 5, n, first=first)
    la, lb = synth.su3(SEED, 0, 4 * n, first=4 * first), synth.su3(SEED, 1, 4 * n, first=4 * first)
    leaves = {"a": a, "b": b, "c": c, "d": d}
    E1 = ("add", ("mul", ("leaf", "a"), ("leaf", "b")), ("mul", ("leaf", "c"), ("leaf", "d")))
    E2 = ("add", ("mul", ("mul", ("leaf", "a"), ("leaf", "b")), ("leaf", "c")),
          ("scale", 0.5, ("leaf", "d")))
    E3 = ("sub", ("mul", ("adj", ("leaf", "a")), ("leaf", "b")),
          ("mul", ("leaf", "b"), ("adj", ("leaf", "a"))))
    MM = ("mul", ("leaf", "a"), ("leaf", "b"))
    bytes_one = n * (B_MM + B_MV + 4 * B_MM + B_E1 + B_E2 + B_E3 + B_F32 + 2 * B_H + B_C12 + B_C12F
                     + B_E1 + B_ADJ_MM + B_ADJ_E1)

    def one_pass():
        oracle.mm(a, b)
        oracle.mv(a, vv)
        oracle.mm(la, lb)
        oracle.eval_tree(E1, leaves)
        oracle.eval_tree(E2, leaves)
        oracle.eval_tree(E3, leaves)
        for fmt in ("f32", "bf16", "f16"):
            oracle.round_to(oracle.mm(oracle.round_to(a, fmt), oracle.round_to(b, fmt)), fmt)
        for fmt in (None, "f32"):
            ra = a[:, :2].copy() if fmt is None else oracle.round_to(a[:, :2].copy(), fmt)
            rb = b[:, :2].copy() if fmt is None else oracle.round_to(b[:, :2].copy(), fmt)
            oracle.mm(oracle.c12_expand(ra), oracle.c12_expand(rb))
        oracle.eval_tree(E1, leaves)   # the batched row: same tree
        oracle.eval_adjoint(MM, leaves, w)
        oracle.eval_adjoint(E1, leaves, w)

    reps, t0 = 0, time.time()
    while True:
        one_pass()
        reps += 1
        if time.time() - t0 >= budget_s:
            break
    return reps * bytes_one, t0, time.time(), reps


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_sample(budget_s=12.0, frac_sites=1 << 16, procs=None):
    """The oracle, as it stands (single-threaded C), on a bounded sample of the
    step, on the host's cores: `procs` spawned processes (default: every core
    this process may use), each running every row's computation on its own
    `frac_sites` sites.  Value: all bytes / (last end - first start)."""
    if procs is None:
        procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 1
    procs = max(1, int(procs))
    jobs = [(k * frac_sites, frac_sites, budget_s) for k in range(procs)]
    if procs == 1:
        res = [_oracle_pass_worker(jobs[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(procs) as pool:   # spawn: no fork after CUDA
            res = pool.map(_oracle_pass_worker, jobs)
    total = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    passes = sum(r[3] for r in res)
    return {"value": total / span / 1e9, "unit": "GB/s", "cores": procs, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": "every row of the step on %d x %d sites (%d processes, %d passes in %.1f s)"
                      % (procs, frac_sites, procs, passes, span),
            "seconds": span, "passes": passes}


# ----------------------------------------------------------------- studies
def _time_ms(torch, stream, fn, reps=20, warm=3):
    for _ in range(warm):
        fn()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    s0.record(stream)
    for _ in range(reps):
        fn()
    s1.record(stream)
    s1.synchronize()
    return s0.elapsed_time(s1) / reps


def run_studies(su3s, synth, torch, stream, which, study_dims=(32, 32, 32, 32)):
    """Measurements the configurations ask for beside the step, one JSON line
    each: the L^4 volume sweep (A2-A4), fused vs term-by-term trees (32^4),
    reduced-precision and two-row storage (32^4 and 16^3x32, with each format's
    stated error bound against the FP64 oracle, which the GPU tests measure),
    batched graph vs separate launches (64 lattices), the layout / site-block
    sweep of z=a*b (the vector-length study of Sec. 5, Fig. 4) and the
    neighbour operations."""
    out = []
    F64, MAT, VEC = su3s.F64, su3s.MATRIX, su3s.VECTOR

    def fld(lat, kind, nmu, prec, arr, layout=su3s.SOA, block=64):
        f = su3s.Field(lat, kind, nmu, prec, layout, block)
        f.upload(arr)
        return f

    if "volume" in which:
        for L in (8, 16, 24, 32, 40, 48):
            dims = (L, L, L, L)
            v = synth.volume(dims)
            lat = su3s.Lattice(dims)
            a = fld(lat, MAT, 1, F64, synth.su3(SEED, 0, v))
            b = fld(lat, MAT, 1, F64, synth.su3(SEED, 1, v))
            x = fld(lat, VEC, 1, F64, synth.gauss_vector(SEED, 4, v))
            la = fld(lat, MAT, 4, F64, synth.su3(SEED, 0, 4 * v))
            lb = fld(lat, MAT, 4, F64, synth.su3(SEED, 1, 4 * v))
            z, zv, zl = a.like(), x.like(), la.like()
            res = {}
            for name, dest, e, bps in (("A2", z, a * b, B_MM), ("A3", zv, a * x, B_MV),
                                       ("A4", zl, la * lb, 4 * B_MM)):
                ms = _time_ms(torch, stream, lambda: su3s.evaluate(dest, e, 0, stream))
                res[name] = {"ms": round(ms, 5), "GB_s": round(bps * v / ms / 1e6, 1),
                             "Gsites_s": round(v / ms / 1e6, 3)}
            # lattices whose fields fit the L2 cache: also time a rotation over
            # enough independent copies of the fields (each evaluation reads
            # the next copy) that their total exceeds twice the L2 size, so
            # every evaluation reads HBM
            rot = {}
            ha, hb, hx = synth.su3(SEED, 0, v), synth.su3(SEED, 1, v), synth.gauss_vector(SEED, 4, v)
            hla, hlb = synth.su3(SEED, 0, 4 * v), synth.su3(SEED, 1, 4 * v)
            for name, bps, mk in (
                    ("A2", B_MM, lambda: (fld(lat, MAT, 1, F64, ha), fld(lat, MAT, 1, F64, hb))),
                    ("A3", B_MV, lambda: (fld(lat, MAT, 1, F64, ha), fld(lat, VEC, 1, F64, hx))),
                    ("A4", 4 * B_MM, lambda: (fld(lat, MAT, 4, F64, hla), fld(lat, MAT, 4, F64, hlb)))):
                set_bytes = bps * v
                if set_bytes >= 2 * 129e6:
                    continue
                nrot = min(256, int(np.ceil(2.4 * 129e6 / set_bytes)))
                sets = []
                for _ in range(nrot):
                    p, q = mk()
                    sets.append((p.like() if name != "A3" else q.like(), p * q, p, q))

                def run_all(sets=sets):
                    for dest, e, _, _ in sets:
                        su3s.evaluate(dest, e, 0, stream)
                ms = _time_ms(torch, stream, run_all, reps=5, warm=2) / nrot
                rot[name] = {"ms": round(ms, 5), "GB_s": round(bps * v / ms / 1e6, 1),
                             "Gsites_s": round(v / ms / 1e6, 3), "copies": nrot}
                del sets
            out.append({"study": "volume sweep", "L": L, "sites": v,
                        "l2_resident": (3 * 144 * v) < 129e6, **res,
                        **({"rotating": rot} if rot else {})})
            del a, b, x, la, lb, z, zv, zl
            torch.cuda.empty_cache()

    if "fused" in which:
        dims = (32, 32, 32, 32)
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        F = {n: fld(lat, MAT, 1, F64, synth.su3(SEED + 1, i, v)) for i, n in enumerate("abcd")}
        a, b, c, d = (F[n] for n in "abcd")
        z, t1, t2 = a.like(), a.like(), a.like()
        for name, fused, steps, fused_b, tbt_b in (
                ("a*b+c*d", a * b + c * d,
                 [(t1, a * b), (t2, c * d), (z, t1 + t2)], B_E1, 3 * 432),
                ("a*b*c+0.5*d", a * b * c + 0.5 * d,
                 [(t1, a * b), (t2, t1 * c), (z, t2 + 0.5 * d)], B_E2, 3 * 432),
                ("adj(a)*b-b*adj(a)", a.adj() * b - b * a.adj(),
                 [(t1, a.adj() * b), (t2, b * a.adj()), (z, t1 - t2)], B_E3, 3 * 432)):
            ms_f = _time_ms(torch, stream, lambda: su3s.evaluate(z, fused, 0, stream))

            def tbt():
                for dst, e in steps:
                    su3s.evaluate(dst, e, 0, stream)
            ms_t = _time_ms(torch, stream, tbt)
            out.append({"study": "fused vs term-by-term", "tree": name, "lattice": list(dims),
                        "fused_ms": round(ms_f, 5), "term_by_term_ms": round(ms_t, 5),
                        "speedup": round(ms_t / ms_f, 3), "fused_B_per_site": fused_b,
                        "term_by_term_B_per_site": tbt_b})
        del F, a, b, c, d, z, t1, t2
        torch.cuda.empty_cache()

    if "precision" in which:
        # the error bounds are the ones the GPU tests assert against the FP64
        # oracle over every output of these lattices (tests/test_gpu_error_study.py)
        fmts = [("f64", F64, 1e-13), ("f32", su3s.F32, 2e-6), ("bf16", su3s.BF16, 2.5e-2),
                ("f16", su3s.F16, 3e-3), ("f64_c12", su3s.F64_C12, 1e-13),
                ("f32_c12", su3s.F32_C12, 5e-6)]
        for dims in ((32, 32, 32, 32), (16, 16, 16, 32)):
            v = synth.volume(dims)
            lat = su3s.Lattice(dims)
            ha, hb = synth.su3(SEED + 2, 0, v), synth.su3(SEED + 2, 1, v)
            for name, prec, bound in fmts:
                a, b = fld(lat, MAT, 1, prec, ha), fld(lat, MAT, 1, prec, hb)
                z = a.like()
                ms = _time_ms(torch, stream, lambda: su3s.evaluate(z, a * b, 0, stream))
                bps = {"f64": B_MM, "f32": B_F32, "bf16": B_H, "f16": B_H, "f64_c12": B_C12,
                       "f32_c12": B_C12F}[name]
                out.append({"study": "precision", "lattice": list(dims), "storage": name,
                            "error_bound_vs_fp64_oracle": bound,
                            "ms": round(ms, 5), "Gsites_s": round(v / ms / 1e6, 3),
                            "GB_s": round(bps * v / ms / 1e6, 1)})
                del a, b, z
            torch.cuda.empty_cache()

    if "interp" in which:
        # trees outside the compiled catalogue run the uniform interpreter
        # kernel (registers in local memory); beside them a catalogue tree of
        # the same byte count for comparison
        dims = (48, 48, 48, 48)
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        F = {n: fld(lat, MAT, 1, F64, synth.su3(SEED + 7, i, v)) for i, n in enumerate("abcd")}
        a, b, c, d = (F[n] for n in "abcd")
        z = a.like()
        cat = {sig for (_, sig, p, m) in su3s.catalogue()}
        for name, e, bsite in (("(a+b)*adj(c)", (a + b) * c.adj(), 4 * 144),
                               ("a*b+c*d (catalogue)", a * b + c * d, 5 * 144),
                               ("a*(b+c)-d", a * (b + c) - d, 5 * 144),
                               ("adj(a*b)*c", (a * b).adj() * c, 4 * 144)):
            for mname in MATH_NAMES:
                ms = _time_ms(torch, stream,
                              lambda: su3s.evaluate(z, e, MATH_IDS[mname], stream))
                out.append({"study": "interpreter", "tree": name, "math": mname,
                            "compiled": e.signature() in cat, "lattice": list(dims),
                            "ms": round(ms, 5), "B_per_site": bsite,
                            "GB_s": round(bsite * v / ms / 1e6, 1)})
        del F, a, b, c, d, z
        torch.cuda.empty_cache()

    if "stencil" in which:
        # nearest-neighbour operations (Sec. 6, Summary and Outlook): the hopping term and the Cshift;
        # algorithmic bytes: every input object once, the output once
        for dims in ((32, 32, 32, 32), (48, 48, 48, 48)):
            v = synth.volume(dims)
            lat = su3s.Lattice(dims)
            U = fld(lat, MAT, 4, F64, synth.su3(SEED + 6, 0, 4 * v))
            for kind, name, bsite in ((su3s.VECTOR, "vector", 576 + 48 + 48),
                                      (MAT, "matrix", 576 + 144 + 144)):
                x = (synth.gauss_vector(SEED + 6, 4, v) if kind == su3s.VECTOR
                     else synth.su3(SEED + 6, 1, v))
                X = fld(lat, kind, 1, F64, x)
                Z = X.like()
                for mname in MATH_NAMES:
                    ms = _time_ms(torch, stream,
                                  lambda: su3s.hop(Z, U, X, MATH_IDS[mname], stream))
                    out.append({"study": "stencil", "op": "hop " + name, "lattice": list(dims),
                                "math": mname, "ms": round(ms, 5), "B_per_site": bsite,
                                "GB_s": round(bsite * v / ms / 1e6, 1),
                                "Gsites_s": round(v / ms / 1e6, 3)})
                del X, Z
            # the Wilson hopping term with spin: spinors are vector fields with
            # 4 spin components; 4 links 576 B + spinor 192 B + output 192 B,
            # 1320 flops per site
            P = fld(lat, su3s.VECTOR, 4, F64, synth.gauss_vector(SEED + 6, 5, 4 * v))
            Q = P.like()
            for mname in MATH_NAMES:
                ms = _time_ms(torch, stream,
                              lambda: su3s.dslash(Q, U, P, MATH_IDS[mname], stream))
                out.append({"study": "stencil", "op": "wilson dslash (spin)", "lattice": list(dims),
                            "math": mname, "ms": round(ms, 5), "B_per_site": 960,
                            "GB_s": round(960 * v / ms / 1e6, 1),
                            "Gsites_s": round(v / ms / 1e6, 3),
                            "GFLOP_s": round(1320 * v / ms / 1e6, 1)})
            del P, Q
            A = fld(lat, MAT, 1, F64, synth.su3(SEED + 6, 2, v))
            B = A.like()
            for dim in (0, 3):
                ms = _time_ms(torch, stream, lambda: su3s.cshift(B, A, dim, 1, stream))
                out.append({"study": "stencil", "op": "cshift matrix dim %d" % dim,
                            "lattice": list(dims), "ms": round(ms, 5), "B_per_site": 288,
                            "GB_s": round(288 * v / ms / 1e6, 1)})
            del U, A, B
            torch.cuda.empty_cache()

    if "hop" in which:
        # the colour hopping term alone on vectors, then on matrices, on the
        # --dims lattice in the default arithmetic (small cases for a profiler)
        dims = study_dims
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        U = fld(lat, MAT, 4, F64, synth.su3(SEED + 6, 0, 4 * v))
        for kind, name, bsite in ((VEC, "vector", 576 + 48 + 48), (MAT, "matrix", 576 + 144 + 144)):
            x = (synth.gauss_vector(SEED + 6, 4, v) if kind == VEC else synth.su3(SEED + 6, 1, v))
            X = fld(lat, kind, 1, F64, x)
            Z = X.like()
            ms = _time_ms(torch, stream, lambda: su3s.hop(Z, U, X, 0, stream), reps=5, warm=2)
            out.append({"study": "hop " + name, "lattice": list(dims), "ms": round(ms, 5),
                        "B_per_site": bsite, "GB_s": round(bsite * v / ms / 1e6, 1)})
            del X, Z
        del U
        torch.cuda.empty_cache()

    if "dslash" in which:
        # the Wilson hopping term with spin alone, on the --dims lattice, in the
        # default arithmetic (a small case for a profiler capture)
        dims = study_dims
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        U = fld(lat, MAT, 4, F64, synth.su3(SEED + 6, 0, 4 * v))
        P = fld(lat, su3s.VECTOR, 4, F64, synth.gauss_vector(SEED + 6, 5, 4 * v))
        Q = P.like()
        ms = _time_ms(torch, stream, lambda: su3s.dslash(Q, U, P, 0, stream), reps=5, warm=2)
        out.append({"study": "wilson dslash (spin)", "lattice": list(dims), "ms": round(ms, 5),
                    "B_per_site": 960, "GB_s": round(960 * v / ms / 1e6, 1)})
        del U, P, Q
        torch.cuda.empty_cache()

    if "blocks" in which:
        # the vector-length / block-shape study of Sec. 5 (Fig. 4 and the 2-d
        # block): z = a*b at 48^4, GB/s against threads per CTA (32-site tiles,
        # i.e. warps, per CTA: the 2-d block's y extent) and CTAs per SM, for
        # the staged and plain-load kernels in FP64 storage (pair arithmetic)
        # and the plain-load kernel in FP32 storage (the paper's single
        # precision).  A CTA of more than 256 threads cannot be resident with
        # these kernels' register use (100-110 per thread), so the sweep ends
        # at 256.
        dims = DIMS
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        ha, hb = synth.su3(SEED, 0, v), synth.su3(SEED, 1, v)
        for prec, pname, pipes, bsite in ((F64, "f64", ((su3s.PIPE_TMA, "tma"), (su3s.PIPE_PLAIN, "plain")), B_MM),
                                          (su3s.F32, "f32", ((su3s.PIPE_PLAIN, "plain"),), 216)):
            a = fld(lat, MAT, 1, prec, ha)
            b = fld(lat, MAT, 1, prec, hb)
            z = a.like()
            for pipe, pipename in pipes:
                su3s.set_pipeline(pipe)
                for threads in (32, 64, 128, 256):
                    for bps in (1, 2, 4, 8, 16, 0):
                        su3s.set_launch(z, a * b, threads, bps)
                        ms = _time_ms(torch, stream, lambda: su3s.evaluate(z, a * b, 0, stream))
                        out.append({"study": "block shape z=a*b", "lattice": list(dims),
                                    "storage": pname, "pipeline": pipename, "threads": threads,
                                    "warps_per_cta": threads // 32,
                                    "ctas_per_sm": bps if bps else "max",
                                    "ms": round(ms, 5), "GB_s": round(bsite * v / ms / 1e6, 1)})
            su3s.set_pipeline(su3s.PIPE_AUTO)
            del a, b, z
            torch.cuda.empty_cache()

    if "batch" in which:
        picks = (synth.uniform_real(SEED + 3, 40, 64) + 1.0) / 2.0 * len(BATCH_SHAPES)
        batch = su3s.Batch()
        items, sites = [], 0
        for i, p in enumerate(picks):
            dims = BATCH_SHAPES[min(int(p), len(BATCH_SHAPES) - 1)]
            lat = su3s.Lattice(dims)
            nv = synth.volume(dims)
            fs = {n: fld(lat, MAT, 1, F64, synth.su3(SEED + 3 + 1000 * i, j, nv))
                  for j, n in enumerate("abcd")}
            zb = fs["a"].like()
            e = fs["a"] * fs["b"] + fs["c"] * fs["d"]
            batch.add(zb, e)
            items.append((lat, fs, zb, e))
            sites += nv
        batch.build()
        ms_g = _time_ms(torch, stream, lambda: batch.launch(stream))

        def separate():
            for _, _, zb, e in items:
                su3s.evaluate(zb, e, 0, stream)
        ms_s = _time_ms(torch, stream, separate)
        out.append({"study": "batched vs separate launches", "lattices": 64, "sites": sites,
                    "graph_ms": round(ms_g, 5), "separate_ms": round(ms_s, 5),
                    "speedup": round(ms_s / ms_g, 3),
                    "graph_GB_s": round(B_E1 * sites / ms_g / 1e6, 1),
                    "separate_GB_s": round(B_E1 * sites / ms_s / 1e6, 1)})
        del batch, items
        torch.cuda.empty_cache()

    if "layout" in which:
        dims = DIMS
        v = synth.volume(dims)
        lat = su3s.Lattice(dims)
        ha, hb = synth.su3(SEED, 0, v), synth.su3(SEED, 1, v)
        for layout, block in ((su3s.SOA, 0), (su3s.AOSOA, 4), (su3s.AOSOA, 16), (su3s.AOSOA, 32),
                              (su3s.AOSOA, 64), (su3s.AOSOA, 128), (su3s.AOSOA, 256),
                              (su3s.AOSOA, 1024)):
            a = fld(lat, MAT, 1, F64, ha, layout, block or 64)
            b = fld(lat, MAT, 1, F64, hb, layout, block or 64)
            z = a.like()
            for pipe, pname in ((su3s.PIPE_PLAIN, "plain"), (su3s.PIPE_TMA, "tma")):
                su3s.set_pipeline(pipe)
                ms = _time_ms(torch, stream, lambda: su3s.evaluate(z, a * b, 0, stream))
                out.append({"study": "layout sweep z=a*b", "lattice": list(dims),
                            "layout": "soa" if layout == su3s.SOA else "aosoa%d" % block,
                            "pipeline": pname, "ms": round(ms, 5),
                            "GB_s": round(B_MM * v / ms / 1e6, 1)})
            su3s.set_pipeline(su3s.PIPE_AUTO)
            del a, b, z
            torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the native-FP64 timings reported beside the step")
    ap.add_argument("--rows", default="",
                    help="comma-separated row-name prefixes to run (default: every row)")
    ap.add_argument("--dims", default="48,48,48,48", help="lattice extents (default 48^4)")
    ap.add_argument("--study", default="",
                    help="comma list of studies to run instead of the step: volume, fused, "
                         "precision, batch, layout, blocks, stencil, interp, hop, dslash (one JSON "
                         "line each; hop and dslash run on the --dims lattice)")
    ap.add_argument("--math", default="df32", choices=["fx", "df32", "f64"],
                    help="arithmetic of the FP64-storage rows in the step (the others are "
                         "timed beside it)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the library's autotuner (by default it picks each row's launch "
                         "shape and data movement during setup, outside the timed region)")
    ap.add_argument("--pipeline", default="auto",
                    choices=["auto", "plain", "tma", "tma_leaf", "tma_ring", "tma_pair"],
                    help="data movement of FP64-storage kernels (default: the library's choice)")
    args = ap.parse_args()
    dims = tuple(int(x) for x in args.dims.split(","))
    if len(dims) == 1:
        dims = dims * 4
    prefixes = [p.strip() for p in args.rows.split(",") if p.strip()]

    def want(name):
        return not prefixes or any(name.startswith(p) for p in prefixes)
    full = not prefixes and dims == DIMS
    ws, rank, local = dist_env()

    if args.impl == "reference":
        if rank != 0:
            return 0
        w_s = 2.0
        k_s = min(25.0, max(5.0, 2.0 * args.steps))
        for _ in range(args.warmup):
            cpu_oracle_sample(budget_s=w_s / max(1, args.warmup), frac_sites=1 << 14)
        cb = cpu_oracle_sample(budget_s=k_s, frac_sites=1 << 16)
        line = {"impl": "reference", "metric": METRIC, "value": round(cb["value"], 4),
                "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "48^4 lattice, every hot-path row (A2-A9), CPU oracle on a "
                                       "bounded sample of sites"},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu")},
                "e2e": {"value": round(cb["value"], 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1710_09409_gb300 as su3s
    import synth
    su3s.load()
    su3s.set_default_math(MATH_IDS[args.math])
    if args.study:
        st = torch.cuda.Stream()
        for line in run_studies(su3s, synth, torch, st, args.study.split(","), dims):
            print(json.dumps(line))
        return 0
    su3s.set_pipeline({"auto": su3s.PIPE_AUTO, "plain": su3s.PIPE_PLAIN, "tma": su3s.PIPE_TMA,
                       "tma_leaf": su3s.PIPE_TMA_LEAF, "tma_ring": su3s.PIPE_TMA_RING,
                       "tma_pair": su3s.PIPE_TMA_PAIR}[args.pipeline])
    stream = torch.cuda.Stream()
    with_host = not args.no_e2e
    e2e_skip = None
    if with_host:
        e2e_skip = e2e_host_shortage(dims, int(os.environ.get("LOCAL_WORLD_SIZE", "1")),
                                     host_mem_available())
        with_host = e2e_skip is None
    rows, keep = build_rows(su3s, synth, torch, with_host, dims, want)
    torch.cuda.synchronize()
    tuned = []
    if not args.no_tune:
        for r in rows:
            if r.tune is not None:
                res = r.tune(stream)
                if isinstance(res, dict):       # the batch: its own launch parameters
                    tuned.append(dict(row=r.name, **res))
                    continue
                th, bps, var, tms = res
                tuned.append({"row": r.name, "threads": th, "blocks_per_sm": bps,
                              "variant": var, "ms": round(tms, 5)})
        torch.cuda.synchronize()

    # device-resident timing
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    total_ms, per_row, launches = time_step(rows, torch, stream, args.steps, args.warmup)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    ms_step = total_ms / args.steps
    bytes_step = sum(r.nbytes for r in rows)
    value = aggregate_gbs(bytes_step, ws, ms_step)

    peak, peak_kind = read_peaks()
    row_out = []
    for r, ms in zip(rows, per_row):
        m = float(np.mean(ms))
        gbs = r.nbytes / (m * 1e-3) / 1e9
        row_out.append({"row": r.name, "storage": r.dtype,
                        "arith": MATH_DTYPE[args.math] if r.dtype.startswith("f64") else "f32",
                        "ms": round(m, 5), "ms_median": round(float(np.median(ms)), 5),
                        "GB_s": round(gbs, 1),
                        "frac_of_peak": round(gbs / peak, 4),
                        "Gsites_s": round(r.sites / (m * 1e-3) / 1e9, 3)})
    # dominant kernel: the kernel with the largest share of the step time,
    # over every row that runs it (rows are grouped by the kernel they launch,
    # as in the launch list); achieved = algorithmic bytes per launch over its
    # average launch time
    variant_of = {t["row"]: t.get("variant") for t in tuned}
    groups = {}
    for r, ms in zip(rows, per_row):
        k, nl, lb = row_launches(r, variant_of.get(r.name))
        g = groups.setdefault(k, {"ms": 0.0, "launches": 0, "bytes": 0.0, "rows": []})
        g["ms"] += float(np.mean(ms))
        g["launches"] += nl
        g["bytes"] += nl * lb
        g["rows"].append(r.name)
    dk = max(groups, key=lambda k: groups[k]["ms"])
    dg = groups[dk]
    per_launch_bytes = dg["bytes"] / dg["launches"]
    per_launch_ms = dg["ms"] / dg["launches"]
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dk, "rows": dg["rows"], "launches_per_step": dg["launches"],
            "share_of_step": round(dg["ms"] / ms_step, 4), "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6800 GB/s",
            "traffic": traffic_bytes(dk, per_launch_bytes),
            "traffic_source": "ncu dram__bytes_read+write per launch at 32^4, scaled by sites",
            "nominal_peak": 7900.0, "frac_nominal": round(achieved / 7900.0, 4),
            "algorithmic_bytes_per_launch": int(round(per_launch_bytes))}
    a2 = row_out[0]

    # the other arithmetics for the FP64 rows, reported beside (not in the step)
    variants = []
    for mname in [m for m in MATH_NAMES if m != args.math]:
        su3s.set_default_math(MATH_IDS[mname])
        for r in (rows if not args.no_variants else []):
            if r.dtype == "f64" and not r.name.startswith("A8"):   # graph fixed at build
                _, pr, _ = time_step([r], torch, stream, 20, 2)
                m = float(np.mean(pr[0]))
                variants.append({"row": r.name, "math": mname, "ms": round(m, 5),
                                 "GB_s": round(r.nbytes / (m * 1e-3) / 1e9, 1)})
    su3s.set_default_math(MATH_IDS[args.math])

    e2e = {"value": None, "unit": "GB/s", "unavailable": e2e_skip} if e2e_skip else None
    if with_host:
        # three runs of the e2e steps: the value is the median run, with the
        # spread beside it; the host link measured on its own bounds the step
        runs = [time_e2e(rows, torch, stream, args.e2e_steps) for _ in range(3)]
        h2d, d2h = runs[0][1], runs[0][2]
        run_ms = sorted(max_over_ranks(r[0], dist, "cuda") for r in runs)
        e_ms = run_ms[1]
        link = measure_link(torch)
        bound_ms = (h2d + d2h) / (link * 1e9) * 1e3
        e2e = {"value": round(aggregate_gbs(bytes_step, ws, e_ms), 2), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e_ms, 3),
               "runs_ms_per_step": [round(x, 3) for x in run_ms],
               "range_GB_s": [round(aggregate_gbs(bytes_step, ws, run_ms[2]), 2),
                              round(aggregate_gbs(bytes_step, ws, run_ms[0]), 2)],
               "host_link_GB_s": round(link, 1),
               "host_link_bound_ms_per_step": round(bound_ms, 3),
               "frac_of_host_link_bound": round(bound_ms / e_ms, 3)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_sample()
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": MATH_DTYPE[args.math], "data": "synthetic",
            "config": {"workload": ("48^4 lattice (5,308,416 sites), every hot-path row A2-A9 once "
                                    "per step; FP64 rows in %s arithmetic" % MATH_DESC[args.math]
                                    if full else "subset %s on %s" % (args.rows or "all rows",
                                                                      "x".join(map(str, dims)))),
                       "storage": "f64 (A2-A5, A7 two-row, A8, A9); f32/bf16/f16 (A6); "
                                  "two-row f32 (A7)",
                       "arithmetic": ("FP64-storage rows in %s, max abs error %s against the FP64 "
                                      "oracle (bound 1e-13); reduced-precision rows in FP32"
                                      % (MATH_DESC[args.math], MATH_ERR[args.math])),
                       "lattice": list(dims), "layout": "soa", "pipeline": args.pipeline,
                       "tuned": not args.no_tune,
                       "l2": "every field larger than the 129 MB L2; no flush needed",
                       "bytes_per_step": bytes_step, "seed": SEED},
            "sites_per_s": round(a2["Gsites_s"] * 1e9 * ws, 0),
            "rows": row_out, "other_arithmetic_rows": variants, "tuned": tuned,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
