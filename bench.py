#!/usr/bin/env python3
"""Throughput of table-free GMM rANS coding on one GB300.

One step = encode + decode of one synthetic latent of 192 x 32 x 48 =
294,912 symbols (a 768 x 512 image at stride 16), K = 3 mixture components
with fp32 parameters, 1024 interleaved rANS streams: per-symbol interval
kernel, rANS encode, offset scan, compaction, then binary-search decode.
Inputs are resident in HBM. The K timed steps run as a coding service runs
them: step i+1's encode (one stream and handle) overlaps step i's decode
(a second stream and handle), and the inputs rotate over 16 buffer sets
that together exceed L2. The same steps one at a time, with L2 flushed
(256 MiB write) before each, are reported under "serial".

Prints one JSON line. `value` is symbols round-tripped (encoded + decoded)
per second, summed over ranks; encode and decode rates are reported beside
it. `--impl reference` times the CPU oracle on the same latent instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="latent_192x32x48_k3_s1024", C=192, H=32, W=48, K=3, S=1024, seed=1002)
# FP32 operations per Phi-hat evaluation, the fixed count of the method's
# arithmetic (1 division, 5 Horner fmaf, exp ~12, clamp/select/accumulate
# ~10); a quantised-CDF evaluation takes K of them. The kernels issue more
# instructions than this (about 34 per component: the reciprocal's Newton
# step, the grid rounding, the exponent scaling and integer conversions are
# separate instructions); the roofline numerator counts the method's work,
# not the instructions.
OPS_PER_PHI = 28
FP32_LANES_PER_SM = 128
# Rotating input sets of the timed loop (more than L2 holds).
ROTATE_SETS = 16
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the decoder the plan names, from the ncu capture of the traffic probe
# (profiles/traffic_roofline_kernels.md); valid for the kernel as captured
# there (null for any other plan).
DECODE_TRAFFIC_BYTES = {"fgmm_dec_ws_kernel/16/4/16": 10793728}   # "kernel/lanes/cluster/round0": bytes per launch
# DRAM bytes per symbol of each roofline row's kernels (K = 3, fp32
# parameters), from the same capture: a launch's bytes divided by its
# symbols; rows multiply by their own symbol count. Other parameter types
# and K were not captured (null).
TRAFFIC_PER_SYMBOL = {
    "encode": 44.55,                       # interval + rANS encode + scan + compaction, one latent
    "fgmm_dec_ws_kernel": 36.65,           # warp-specialised decoder
    "batch_encode": 40.68,                 # fgmm_batch_enc_kt_kernel + scan + batch compaction
    "fgmm_batch_dec_kt_kernel": 38.48,     # batch decoder
    "fgmm_batch_dec_prop_kernel": 38.26,   # batched proposal decoder
}
TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of bench.py --traffic-probe"


def ops_per_eval(K: int) -> int:
    """FP32 operations of one quantised-CDF evaluation (K Phi-hat)."""
    return OPS_PER_PHI * K


def slot_bytes(N: int, K: int, S: int) -> int:
    """Device bytes of one input/output set of the timed loop: fp32
    parameters, symbols, the encode bound of words, offsets, decoded
    symbols."""
    T = -(-N // S)
    cap = (S // 32) * (3 * 32 * T + 64)
    return 3 * K * N * 4 + 4 * N + 2 * cap + 8 * (S // 32 + 1) + 4 * N


def workload_config(N: int, K: int, S: int) -> dict:
    """The config dict both arms print (same workload, same keys)."""
    return {"workload": WORKLOAD["name"], "symbols": N, "K": K, "S": S, "params": "fp32",
            "l2": f"inputs larger than L2: {ROTATE_SETS} rotating buffer sets, "
                  f"{ROTATE_SETS * slot_bytes(N, K, S) / 1e6:.0f} MB"}


def host_cpu():
    """Core count and CPU model of this host."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    info = {}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip(), v.strip())
    except Exception:
        pass
    model = info.get("Model name")
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": cores, "model": model or "unknown", "vendor": info.get("Vendor ID", "unknown"),
            "machine": os.uname().machine}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fgmm", choices=["fgmm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--e2e-buffers", type=int, default=3, help="buffer sets of the pipelined end-to-end loop")
    ap.add_argument("--decode-lanes", type=int, default=0, help="0 = automatic")
    ap.add_argument("--no-throughput", action="store_true", help="skip the large-workload section")
    ap.add_argument("--batch-only", type=int, default=0, metavar="N",
                    help="run only the batch case on the first N latents of the 64-latent batch (for profiling)")
    ap.add_argument("--gsm-only", action="store_true",
                    help="run only the Gaussian-single-model case (for profiling its decoder)")
    ap.add_argument("--proposal-only", action="store_true",
                    help="run only the learned-proposal case (for profiling its decoders)")
    ap.add_argument("--proposal-latents", type=int, default=16, help="latents decoded in --proposal-only mode")
    ap.add_argument("--traffic-probe", action="store_true",
                    help="launch each roofline kernel twice on small cases, for an ncu capture of DRAM bytes")
    ap.add_argument("--proposal-train-scale", type=float, default=1.0,
                    help="fraction of the training schedule in --proposal-only mode")
    ap.add_argument("--ckbd-only", action="store_true",
                    help="run only the checkerboard two-pass case (for profiling its fused decoder)")
    ap.add_argument("--batch-table", action="store_true",
                    help="in --batch-only mode, also time the table-based coder on the batch in chunks")
    ap.add_argument("--batch-overhead", type=float, default=0.01,
                    help="container-overhead bound given to the stream autotuner in --batch-only mode")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.gpu)], stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_round_trips(lat, S, threads, budget_s):
    """Encode + decode round trips of the whole latent with the oracle on
    `threads` host threads (segments spread over them), until budget_s has
    passed; returns (round trips, seconds)."""
    import oracle
    t0 = time.perf_counter()
    reps = 0
    while True:
        words, offsets = oracle.encode(lat.params, lat.symbols, S, threads=threads)
        out, st = oracle.decode(lat.params, words, offsets, S, threads=threads)
        assert st == 0
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    return reps, time.perf_counter() - t0


def cpu_baseline(lat, S, budget_s=6.0):
    """The CPU oracle, as it stands, on the same latent: on all host cores
    (its segments spread over one thread per core) and on one thread."""
    host = host_cpu()
    n = host["nproc"]
    r1, t1 = _oracle_round_trips(lat, S, 1, budget_s)
    rn, tn = _oracle_round_trips(lat, S, n, budget_s)
    return {"value": rn * lat.N / tn / 1e6, "unit": "Msymbols/s", "cores": n, "kind": "oracle",
            "sample": f"{rn} encode+decode round trip(s) of the full {lat.N}-symbol latent, segments over {n} threads",
            "single_thread": {"value": r1 * lat.N / t1 / 1e6, "unit": "Msymbols/s", "cores": 1,
                              "sample": f"{r1} round trip(s) of the full latent on one thread"},
            "host": host}


def _events_ms(fn, reps, flush=None):
    """Median CUDA-event time of fn over reps runs, after one untimed run
    (first-launch costs such as a graph's upload stay out)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for i in range(reps):
        if flush is not None:
            flush.fill_(i & 0xff)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_alu_peaks(dev, h, reps=5):
    """Measured FP32 FMA and XU reciprocal throughput of this GPU, in
    T lane-ops/s: the library's throughput probe (independent instruction
    chains on every SM) timed with CUDA events on its stream."""
    import torch
    from paper_2509_18815_gb300 import _abi, codec
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    res = {}
    # about a millisecond per launch, so that launch overhead does not count
    for name, kind, iters in (("fma", _abi.FGMM_PEAK_FMA, 2048), ("rcp", _abi.FGMM_PEAK_RCP, 256)):
        ops = [0.0]

        def run():
            ops[0] = codec.peak_probe(kind, iters, sink, h)

        for _ in range(3):
            run()
        ms = _events_ms(run, reps)
        res[name] = ops[0] / (ms * 1e-3) / 1e12
    return res


def table_batch(dev, h, b, params, syms):
    """The table-based comparison coder on a batch, in chunks of one latent
    (its table, 1 KB per symbol, built for that latent alone and reused for
    the next): per latent the table build + table-driven encode, then the
    table build + table search decode, each launched on one stream; the
    stream of every latent is asserted identical to the table-free batch's.
    Returns total device time per direction (CUDA events around the whole
    chunk loop)."""
    import torch
    from paper_2509_18815_gb300 import _abi, codec
    import ctypes
    nmax = max(int(p.shape[2]) for p in params)
    table = torch.empty((nmax, 512), dtype=torch.int16, device=dev)
    capmax = max(codec.encode_bound_words(int(p.shape[2]), S) for p, S in zip(params, b.S))
    words = torch.empty(capmax, dtype=torch.int16, device=dev)
    offsets = torch.empty(max(S // 32 for S in b.S) + 1, dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    outs = torch.empty(nmax, dtype=torch.int32, device=dev)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    descs = [codec.latent(p) for p in params]
    streams = [b.latent_stream(i) for i in range(len(params))]

    def enc_all(check=False):
        for i, (p, y, S) in enumerate(zip(params, syms, b.S)):
            cap = codec.encode_bound_words(int(p.shape[2]), S)
            h.check(_abi.fgmm_table_encode(h.ptr, ctypes.byref(descs[i]), y.data_ptr(), S, table.data_ptr(),
                                           words.data_ptr(), cap, offsets.data_ptr(), total.data_ptr(), sp))
            if check:
                h.sync()
                w_ref, o_ref = streams[i]
                nw = int(total.item())
                assert nw == w_ref.numel() and torch.equal(words[:nw], w_ref), f"table stream differs (latent {i})"
                assert torch.equal(offsets[: S // 32 + 1], o_ref)

    def dec_all(check=False):
        for i, (p, y, S) in enumerate(zip(params, syms, b.S)):
            w_ref, o_ref = streams[i]
            n = int(p.shape[2])
            h.check(_abi.fgmm_table_decode(h.ptr, ctypes.byref(descs[i]), table.data_ptr(), w_ref.data_ptr(),
                                           w_ref.numel(), o_ref.data_ptr(), S, outs.data_ptr(), sp))
            if check:
                h.sync()
                assert torch.equal(outs[:n], y), f"table decode differs (latent {i})"

    enc_all(check=True)
    dec_all(check=True)
    te = _events_ms(enc_all, 2)
    td = _events_ms(dec_all, 2)
    h.sync()
    del table
    return te, td, nmax * 512 * 2


def batch_case(dev, h, out, name, lats, alu_peak_tops, hbm_gbs, reps=10, max_overhead=0.01, table=False):
    """Batch of latents: one persistent launch per direction replayed from a
    CUDA graph, autotuned streams per latent; adds out[name]. table: also
    time the table-based comparison coder on the same batch."""
    import torch
    from paper_2509_18815_gb300 import codec
    params = [torch.from_numpy(l.params).to(dev) for l in lats]
    syms = [torch.from_numpy(l.symbols).to(dev) for l in lats]
    N = sum(l.N for l in lats)
    b = codec.Batch(params, syms, S=codec.autotune([l.N for l in lats], max_overhead=max_overhead, h=h), h=h)
    b.capture()
    b.encode()
    b.decode()
    assert all(torch.equal(b.decoded[i], syms[i]) for i in range(len(lats))), name
    nw = int(b.total.item())
    codec.stats_enable(True, h); codec.stats_read(h)
    b.decode()
    evals, _ = codec.stats_read(h)
    codec.stats_enable(False, h)
    te = _events_ms(lambda: b.encode(sync=False), reps)
    td = _events_ms(lambda: b.decode(sync=False), reps)
    coded = 0.0
    for p_, s_ in zip(params, syms):
        coded += codec.rate_audit(p_, s_, h)[1]
    tab = table_batch(dev, h, b, params, syms) if table else None
    b.close()
    bytes_sym = 36.0 + 4.0 + 16.0 * nw / N / 8.0
    enc_ops = 2 * N * ops_per_eval(3)
    dec_ops = evals * ops_per_eval(3)
    out[name] = {
        "symbols": N, "latents": len(lats), "segments": sum(s // 32 for s in b.S),
        "encode_msym_s": N / te / 1e3, "decode_msym_s": N / td / 1e3, "ms_encode": te, "ms_decode": td,
        "container_overhead_pct": 100.0 * (16.0 * nw / coded - 1.0),
        "encode_roofline": {"hbm_frac": N * bytes_sym / (te * 1e-3) / 1e9 / hbm_gbs,
                            "alu_frac": enc_ops / (te * 1e-3) / 1e12 / alu_peak_tops,
                            "traffic": TRAFFIC_PER_SYMBOL["batch_encode"] * N},
        "decode_roofline": {"alu_frac": dec_ops / (td * 1e-3) / 1e12 / alu_peak_tops,
                            "hbm_frac": N * bytes_sym / (td * 1e-3) / 1e9 / hbm_gbs,
                            "traffic": TRAFFIC_PER_SYMBOL["fgmm_batch_dec_kt_kernel"] * N},
        "traffic_source": TRAFFIC_SOURCE,
        "ops_per_cdf_eval": ops_per_eval(3), "cdf_evals_per_symbol": evals / N,
    }
    if tab is not None:
        tte, ttd, tbytes = tab
        out[name]["table_coder"] = {
            "encode_msym_s": N / tte / 1e3, "decode_msym_s": N / ttd / 1e3, "ms_encode": tte, "ms_decode": ttd,
            "encode_speedup_table_free": tte / te, "decode_speedup_table_free": ttd / td,
            "chunks": len(lats), "table_mb_per_chunk_max": tbytes / 1e6, "stream_identical": True,
            "schedule": "one latent per chunk: table build + table-driven coding per latent, launched back to back"}
    del params, syms


def gsm_case(dev, h, flush, reps):
    """Gaussian single model with 64 pre-built level tables (Sec. II-C)
    against the table-free coder on the same residuals with the exact scale
    (K = 1), on a 320x64x96 latent of residuals: time per direction (the
    decoder includes its level pre-pass), and rate against the FP64 ideal of
    the exact scale."""
    import numpy as np
    import torch
    from paper_2509_18815_gb300 import codec, synth
    lat = synth.make_gsm_latent(320, 64, 96, seed=1003)
    N = lat.N
    dsg = torch.from_numpy(lat.scales).to(dev)
    dq = torch.from_numpy(lat.symbols).to(dev)
    exact = torch.stack([torch.ones_like(dsg), torch.zeros_like(dsg), dsg])[:, None, :].contiguous()
    blob = codec.gsm_build(device=dev, h=h)
    t_build = _events_ms(lambda: codec.gsm_build(device=dev, h=h), reps)
    ideal, coded_k1, _, _ = codec.rate_audit(exact, dq, h)
    sf = codec.gsm_freqs(dsg, dq, blob, h).to(torch.int64) & 0xffffffff
    fr = (sf >> 16).to(torch.float64)
    esc = ((sf & 0xffff) + (sf >> 16)) == 65536
    coded_gsm = float((16.0 - torch.log2(fr)).sum().item()) + 32.0 * int(esc.sum().item())
    res = {"symbols": N, "levels": 64, "tables_bytes": blob.numel(), "ms_build_tables": t_build,
           "ideal_bits_per_symbol": ideal / N,
           "gsm_overhead_pct": 100.0 * (coded_gsm / ideal - 1.0),
           "table_free_k1_overhead_pct": 100.0 * (coded_k1 / ideal - 1.0), "by_streams": []}
    out = torch.empty(N, dtype=torch.int32, device=dev)
    for S in (1024, codec.autotune([N], bits_per_symbol=ideal / N, h=h)[0], 16384):
        w, o = codec.gsm_encode(dsg, dq, S, blob, h=h)
        codec.gsm_decode(dsg, w, o, S, blob, h=h, out=out)
        assert torch.equal(out, dq)
        te = _events_ms(lambda: codec.gsm_encode(dsg, dq, S, blob, h=h, sync=False), reps, flush)
        td = _events_ms(lambda: codec.gsm_decode(dsg, w, o, S, blob, h=h, out=out, sync=False), reps, flush)
        w1, o1 = codec.encode(exact, dq, S, h=h)
        codec.decode(exact, w1, o1, S, h=h, out=out)
        assert torch.equal(out, dq)
        te1 = _events_ms(lambda: codec.encode(exact, dq, S, h=h, sync=False), reps, flush)
        td1 = _events_ms(lambda: codec.decode(exact, w1, o1, S, h=h, out=out, sync=False), reps, flush)
        res["by_streams"].append({
            "S": S, "gsm": {"encode_msym_s": N / te / 1e3, "decode_msym_s": N / td / 1e3, "ms_encode": te,
                            "ms_decode": td, "bits_per_symbol": 16.0 * w.numel() / N},
            "table_free_k1": {"encode_msym_s": N / te1 / 1e3, "decode_msym_s": N / td1 / 1e3, "ms_encode": te1,
                              "ms_decode": td1, "bits_per_symbol": 16.0 * w1.numel() / N,
                              "decoder": codec.decode_plan(S, h=h)}})
        del w, o, w1, o1
    return res


def ckbd_case(dev, h, flush, reps):
    """Checkerboard two-pass coding (anchors, then the non-anchors with the
    stand-in context's parameters) of the 192x32x48 K = 3 latent with 512
    streams per pass (288 steps each, as the one-pass headline at 1024):
    time per direction including split, context and merge (decode: the
    fused two-pass launch and, for comparison, the separate calls), and the
    rate of both passes against one pass with the hyperprior's parameters."""
    import torch
    from paper_2509_18815_gb300 import codec, synth
    shape = (192, 32, 48)
    lat = synth.make_ckbd_latent(*shape, 3, seed=1002)
    N = lat.N
    dp = torch.from_numpy(lat.params).to(dev)
    dy = torch.from_numpy(lat.symbols).to(dev)
    Sa = Sn = 512
    first, second = codec.ckbd_encode(dp, dy, shape, Sa, Sn, h=h)
    y = codec.ckbd_decode(dp, first, second, shape, Sa, Sn, h=h)
    assert torch.equal(y, dy)
    te_host = _events_ms(lambda: codec.ckbd_encode(dp, dy, shape, Sa, Sn, h=h), reps, flush)
    td_host = _events_ms(lambda: codec.ckbd_decode(dp, first, second, shape, Sa, Sn, h=h, sync=False), reps, flush)
    # the same sequences captured once into CUDA graphs and replayed
    gr = codec.CkbdGraphs(dp, shape, Sa, Sn, h=h)
    gr.capture_encode(dy)
    (wa, oa, ta), (wn, on, tn) = gr.encode()
    assert torch.equal(wa[: int(ta.item())], first[0]) and torch.equal(wn[: int(tn.item())], second[0])
    gr.capture_decode(first, second)
    assert torch.equal(gr.decode(), dy)
    te = _events_ms(lambda: gr.encode(sync=False), reps, flush)
    td = _events_ms(lambda: gr.decode(sync=False), reps, flush)
    h.sync()
    fused = codec.ckbd_decode_fused(3, torch.float32, shape, Sa, Sn, h=h)
    # the same decode as its separate calls (split, pass 1, merge, context,
    # pass 2, merge), captured into a graph too
    y_s = codec.ckbd_decode_steps(dp, first, second, shape, Sa, Sn, h=h)
    assert torch.equal(y_s, dy)
    g_s = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_s, capture_error_mode="thread_local"):
        y_s = codec.ckbd_decode_steps(dp, first, second, shape, Sa, Sn, h=h, sync=False)
    g_s.replay()
    h.sync()
    assert torch.equal(y_s, dy)
    td_steps = _events_ms(lambda: g_s.replay(), reps, flush)
    h.sync()
    # the encode as its separate calls (split, context, two encodes), in a graph
    g_e = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_e, capture_error_mode="thread_local"):
        enc_s = codec.ckbd_encode_steps(dp, dy, shape, Sa, Sn, h=h, sync=False)
    g_e.replay()
    h.sync()
    assert torch.equal(enc_s[0][0][: int(enc_s[0][2].item())], first[0])
    assert torch.equal(enc_s[1][0][: int(enc_s[1][2].item())], second[0])
    te_steps = _events_ms(lambda: g_e.replay(), reps, flush)
    h.sync()
    w1, o1 = codec.encode(dp, dy, 1024, h=h)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    td1 = _events_ms(lambda: codec.decode(dp, w1, o1, 1024, h=h, out=out, sync=False), reps, flush)
    ideal1, _, _, _ = codec.rate_audit(dp, dy, h)
    pa, ya, _, yn = codec.ckbd_split(dp, dy, shape, h)
    pn = codec.ckbd_context(dp, dy, shape, h=h)
    ia, _, _, _ = codec.rate_audit(pa, ya, h)
    inn, _, _, _ = codec.rate_audit(pn, yn, h)
    bits2 = 16.0 * (first[0].numel() + second[0].numel())
    return {"symbols": N, "S_per_pass": [Sa, Sn], "ms_encode": te, "ms_decode": td,
            "encode_msym_s": N / te / 1e3, "decode_msym_s": N / td / 1e3, "one_pass_ms_decode": td1,
            "decode_fused": fused, "ms_decode_separate_calls": td_steps, "ms_encode_separate_calls": te_steps,
            "host_launched": {"ms_encode": te_host, "ms_decode": td_host},
            "ideal_bits_per_symbol_one_pass": ideal1 / N, "ideal_bits_per_symbol_two_pass": (ia + inn) / N,
            "coded_bits_per_symbol_two_pass": bits2 / N,
            "note": "each direction replayed from one CUDA graph: encode = fgmm_ckbd_encode (both passes' "
                    "intervals with split and context in one kernel, both rANS encoders in one launch, scans, "
                    "compactions); decode = fgmm_ckbd_decode (split, both passes in one launch with the context "
                    "applied as pass 2 loads its parameters, merge); *_separate_calls: split, context and two "
                    "encodes / split, pass 1, merge, context, pass 2, merge as separate launches in a graph "
                    "(host_launched: the one-call entries launched from the host)"}


def proposal_case(dev, h, alu_peak_tops, reps=3, n_train=10_000_000, n_latents=16, train_scale=1.0):
    """The learned decode proposal on its workload: the network trained on
    n_train (params, slot, symbol) triples drawn from synthetic latents with
    scales up to 64 (slots uniform inside each symbol's interval), once with
    each activation; then a batch of 16 latents of 320x64x96 (scales up to
    64), autotuned streams, decoded in one persistent launch each by the
    plain batch decoder (graph replay), the network proposal (both
    activations) and the analytic proposal. Every arm's roofline fraction
    uses the same algorithmic work: the plain binary search's CDF
    evaluations x the fixed operation count."""
    import numpy as np
    import torch
    from paper_2509_18815_gb300 import _abi, codec, synth
    from paper_2509_18815_gb300.proposal import init_theta
    train = synth.make_latent(160, 256, 256, 3, seed=1005, sigma_max=64.0)
    ntr = min(n_train, train.N)
    tp = torch.from_numpy(np.ascontiguousarray(train.params[:, :, :ntr])).to(dev)
    ty = torch.from_numpy(np.ascontiguousarray(train.symbols[:ntr])).to(dev)
    rng = np.random.default_rng(11)
    X, t = codec.mlp_data(tp, ty, torch.from_numpy(rng.random(ntr).astype(np.float32)).to(dev), h)
    del tp, ty
    schedule = [(max(1, int(st * train_scale)), lr) for st, lr in [(6000, 3e-3), (3000, 1e-3), (3000, 3e-4)]]
    packed, train_s, final_loss = {}, {}, {}
    for name, act in (("pl", _abi.FGMM_MLP_ACT_PL), ("sigmoid", _abi.FGMM_MLP_ACT_SIGMOID)):
        codec.set_mlp_act(act, h)
        tr = codec.MlpTrainer(init_theta(12), device=dev, h=h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for steps, lr in schedule:
            trace = tr.train(X, t, steps=steps, batch=8192, lr=lr)
        train_s[name] = time.perf_counter() - t0
        final_loss[name] = float(trace[-200:].mean().item())
        packed[name] = tr.packed()
    codec.set_mlp_act(_abi.FGMM_MLP_ACT_PL, h)
    del X, t
    lats = [synth.make_latent(320, 64, 96, 3, seed=1105 + i, sigma_max=64.0) for i in range(n_latents)]
    params = [torch.from_numpy(l.params).to(dev) for l in lats]
    syms = [torch.from_numpy(l.symbols).to(dev) for l in lats]
    N = sum(l.N for l in lats)
    b = codec.Batch(params, syms, S=codec.autotune([l.N for l in lats], h=h), h=h)
    b.capture()
    b.encode()
    arms = {"plain": (lambda: b.decode(sync=False), _abi.FGMM_MLP_ACT_PL),
            "proposal_pl": (lambda: b.decode_proposal(packed["pl"], sync=False), _abi.FGMM_MLP_ACT_PL),
            "proposal_sigmoid": (lambda: b.decode_proposal(packed["sigmoid"], sync=False),
                                 _abi.FGMM_MLP_ACT_SIGMOID),
            "analytic": (lambda: b.decode_proposal(None, sync=False), _abi.FGMM_MLP_ACT_PL)}
    res = {}
    for name, (fn, act) in arms.items():
        codec.set_mlp_act(act, h)
        for d in b.decoded:
            d.zero_()
        codec.stats_enable(True, h); codec.stats_read(h)
        fn(); h.sync()
        probes, nd, hits, fb = codec.stats_read(h, with_hits=True, with_fallbacks=True)
        codec.stats_enable(False, h)
        assert nd == N and all(torch.equal(b.decoded[i], syms[i]) for i in range(len(lats))), name
        ms = _events_ms(fn, reps)
        res[name] = {"ms_decode": ms, "decode_msym_s": N / ms / 1e3, "probes_per_symbol": probes / N,
                     "hit_rate": hits / N if name != "plain" else None, "exact_fallbacks": fb}
    codec.set_mlp_act(_abi.FGMM_MLP_ACT_PL, h)
    b.close()
    evals_plain = res["plain"]["probes_per_symbol"] * N   # the binary search's CDF evaluations
    for name, r in res.items():
        r["alu_frac"] = evals_plain * ops_per_eval(3) / (r["ms_decode"] * 1e-3) / 1e12 / alu_peak_tops
        r["traffic"] = TRAFFIC_PER_SYMBOL["fgmm_batch_dec_kt_kernel" if name == "plain" else
                                          "fgmm_batch_dec_prop_kernel"] * N
    return {"symbols": N, "latents": len(lats), "streams_per_latent": b.S[0], "segments": b.seg_base[-1],
            "train_triples": ntr, "train_steps": sum(st for st, _ in schedule), "train_batch": 8192,
            "train_s": train_s, "train_final_loss": final_loss, "arms": res,
            "note": "one persistent launch per arm over all 16 latents; the plain arm is the batch decoder "
                    "(binary search steered by the fast CDF, confirmed exactly); the proposal arms search from "
                    "the network's guess with the same fast probes and exact confirmation"}


def throughput_workloads(dev, alu_peak_tops, hbm_gbs, reps=10):
    """Larger workloads: one 320x64x96 latent (K = 3 and 4, fp32 and bf16
    parameters, autotuned stream count, FP64 rate audit), a batch of 64
    uneven K = 3 latents (one persistent launch per direction replayed from a
    CUDA graph), and the learned proposal on 16 latents with scales up to
    64. Inputs exceed L2 or L2 is flushed between runs."""
    import numpy as np
    import torch
    from paper_2509_18815_gb300 import _abi, codec, synth
    h = codec.handle(dev)
    out = {}

    # one latent of 320 x 64 x 96: autotuned S, single-latent encode / decode
    # (automatic decoder configuration), K = 3 and 4, fp32 and bf16
    # parameters, with the FP64 rate audit and the roofline fractions
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for K3, bf16 in [(3, False), (4, False), (3, True), (4, True)]:
        lat3 = synth.make_latent(320, 64, 96, K3, 1003)
        if bf16:
            dp3 = torch.from_numpy(synth.to_bf16_bits(lat3.params).view(np.int16)).to(dev).view(torch.bfloat16)
        else:
            dp3 = torch.from_numpy(lat3.params).to(dev)
        ds3 = torch.from_numpy(lat3.symbols).to(dev)
        S3 = codec.autotune([lat3.N], h=h)[0]
        w3, o3 = codec.encode(dp3, ds3, S3, h=h)
        out3 = torch.empty(lat3.N, dtype=torch.int32, device=dev)
        codec.decode(dp3, w3, o3, S3, h=h, out=out3)
        assert torch.equal(out3, ds3)
        # binary-search CDF evaluations (one lane per stream) for the roofline
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 1))
        codec.stats_enable(True, h); codec.stats_read(h)
        codec.decode(dp3, w3, o3, S3, h=h, out=out3)
        evals3, _ = codec.stats_read(h)
        codec.stats_enable(False, h)
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 0))
        te3 = _events_ms(lambda: codec.encode(dp3, ds3, S3, h=h, sync=False), reps, flush)
        td3 = _events_ms(lambda: codec.decode(dp3, w3, o3, S3, h=h, out=out3, sync=False), reps, flush)
        ideal3, coded3, maxerr3, nesc3 = codec.rate_audit(dp3, ds3, h)
        N3 = lat3.N
        ops_eval = ops_per_eval(K3)
        bytes_sym = 3 * K3 * (2 if bf16 else 4) + 4 + 16.0 * w3.numel() / N3 / 8.0
        out[f"latent_320x64x96_k{K3}_{'bf16' if bf16 else 'fp32'}"] = {
            "symbols": N3, "S": S3, "segments": S3 // 32, "decoder": codec.decode_plan(S3, h=h),
            "encode_msym_s": N3 / te3 / 1e3, "decode_msym_s": N3 / td3 / 1e3, "ms_encode": te3, "ms_decode": td3,
            "overhead_pct": 100.0 * (coded3 / ideal3 - 1.0), "max_cdf_err": maxerr3, "escapes": nesc3,
            "container_overhead_pct": 100.0 * (16.0 * w3.numel() / coded3 - 1.0),
            "encode_roofline": {"hbm_frac": N3 * bytes_sym / (te3 * 1e-3) / 1e9 / hbm_gbs,
                                "alu_frac": 2 * N3 * ops_eval / (te3 * 1e-3) / 1e12 / alu_peak_tops,
                                "traffic": (TRAFFIC_PER_SYMBOL["encode"] * N3) if (K3 == 3 and not bf16) else None},
            "decode_roofline": {"alu_frac": evals3 * ops_eval / (td3 * 1e-3) / 1e12 / alu_peak_tops,
                                "cdf_evals_per_symbol": evals3 / N3,
                                "traffic": (TRAFFIC_PER_SYMBOL["fgmm_dec_ws_kernel"] * N3)
                                if (K3 == 3 and not bf16 and codec.decode_plan(S3, h=h)["kernel"] == "fgmm_dec_ws_kernel")
                                else None},
            "traffic_source": TRAFFIC_SOURCE,
        }
        del dp3, ds3, w3, o3, out3
    # the autotuner's trade-off on the K = 3 fp32 latent: a looser bound on
    # the container overhead buys more streams
    lat3 = synth.make_latent(320, 64, 96, 3, 1003)
    dp3 = torch.from_numpy(lat3.params).to(dev)
    ds3 = torch.from_numpy(lat3.symbols).to(dev)
    ideal3, _, _, _ = codec.rate_audit(dp3, ds3, h)
    trade = []
    for ovh in (0.01, 0.03, 0.1, 0.3):
        S3 = codec.autotune([lat3.N], max_overhead=ovh, h=h)[0]
        w3, o3 = codec.encode(dp3, ds3, S3, h=h)
        out3 = torch.empty(lat3.N, dtype=torch.int32, device=dev)
        codec.decode(dp3, w3, o3, S3, h=h, out=out3)
        assert torch.equal(out3, ds3)
        te3 = _events_ms(lambda: codec.encode(dp3, ds3, S3, h=h, sync=False), reps, flush)
        td3 = _events_ms(lambda: codec.decode(dp3, w3, o3, S3, h=h, out=out3, sync=False), reps, flush)
        trade.append({"max_overhead": ovh, "S": S3, "decoder": codec.decode_plan(S3, h=h),
                      "bits_per_symbol": 16.0 * w3.numel() / lat3.N,
                      "total_overhead_pct": 100.0 * (16.0 * w3.numel() / ideal3 - 1.0),
                      "encode_msym_s": lat3.N / te3 / 1e3, "decode_msym_s": lat3.N / td3 / 1e3})
        del w3, o3, out3
    out["latent_320x64x96_k3_fp32_streams_tradeoff"] = trade
    del dp3, ds3
    out["gsm_320x64x96"] = gsm_case(dev, h, flush, reps)
    out["ckbd_192x32x48_k3"] = ckbd_case(dev, h, flush, reps)
    del flush
    shapes = synth.batch_shapes(64, seed=1004)
    batch_case(dev, h, out, "batch64_uneven_k3",
               [synth.make_latent(C, H, W, 3, 1004 + i) for i, (C, H, W) in enumerate(shapes)], alu_peak_tops,
               hbm_gbs, reps, table=True)

    out["proposal_16x320x64x96_sigma64"] = proposal_case(dev, h, alu_peak_tops, reps=reps)
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on all host cores, one
    encode + decode of the full headline latent per step; the one-thread
    figure is reported beside it."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2509_18815_gb300 import synth
    import oracle
    oracle.build()
    lat = synth.make_latent(WORKLOAD["C"], WORKLOAD["H"], WORKLOAD["W"], WORKLOAD["K"], WORKLOAD["seed"])
    S = WORKLOAD["S"]
    host = host_cpu()
    threads = host["nproc"]
    for _ in range(args.warmup):
        w, o = oracle.encode(lat.params, lat.symbols, S, threads=threads)
        oracle.decode(lat.params, w, o, S, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        w, o = oracle.encode(lat.params, lat.symbols, S, threads=threads)
        out, st = oracle.decode(lat.params, w, o, S, threads=threads)
        times.append(time.perf_counter() - t0)
        assert st == 0
    ms = 1e3 * sum(times) / len(times)
    value = lat.N / (ms * 1e-3) / 1e6
    r1, t1 = _oracle_round_trips(lat, S, 1, 2.0)
    print(json.dumps({
        "impl": "reference", "metric": "encode+decode Msymbols/s (round trip)", "value": value,
        "unit": "Msymbols/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(lat.N, WORKLOAD["K"], S),
        "cpu_baseline": {"value": value, "unit": "Msymbols/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step one encode+decode of the full {lat.N}-symbol latent, "
                                   f"segments over {threads} threads",
                         "single_thread": {"value": r1 * lat.N / t1 / 1e6, "unit": "Msymbols/s", "cores": 1,
                                           "sample": f"{r1} round trip(s) of the full latent on one thread"},
                         "host": host},
        "e2e": {"value": value, "unit": "Msymbols/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_fgmm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2509_18815_gb300 import _abi, build, codec, synth
    from paper_2509_18815_gb300.dist import max_over_ranks
    build.build()
    import ctypes

    lat = synth.make_latent(WORKLOAD["C"], WORKLOAD["H"], WORKLOAD["W"], WORKLOAD["K"], WORKLOAD["seed"])
    S, N, K = WORKLOAD["S"], lat.N, WORKLOAD["K"]
    dev = torch.device("cuda", local)
    dp = torch.from_numpy(lat.params).to(dev)
    ds = torch.from_numpy(lat.symbols).to(dev)
    h = codec.handle(dev)
    desc = codec.latent(dp)
    cap = codec.encode_bound_words(N, S)
    words = torch.empty(cap, dtype=torch.int16, device=dev)
    offsets = torch.empty(S // 32 + 1, dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    L = ctypes.byref(desc)

    def enc():
        h.check(_abi.fgmm_encode(h.ptr, L, ds.data_ptr(), S, words.data_ptr(), cap, offsets.data_ptr(),
                                 total.data_ptr(), sptr))

    def dec():
        h.check(_abi.fgmm_decode(h.ptr, L, words.data_ptr(), cap, offsets.data_ptr(), S, out.data_ptr(), sptr))

    # interval, rANS encode, scan and compaction (one launch up to 1,024
    # segments, else two); decode
    launches_per_step = (3 if S // 32 <= 1024 else 4) + 1
    alu_peaks = measure_alu_peaks(dev, h)

    # correctness gate and algorithmic work (CDF evaluations) outside timing
    enc(); dec(); h.sync()
    assert torch.equal(out.cpu(), ds.cpu()), "round trip failed"
    n_words = int(total.item())
    # algorithmic work: CDF evaluations of the plain binary search (one lane
    # per stream); the timed decoder may evaluate more points per round
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 1))
    codec.stats_enable(True, h); codec.stats_read(h)
    dec(); h.sync()
    cdf_evals, nsym = codec.stats_read(h)
    codec.stats_enable(False, h)
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, args.decode_lanes))
    dec(); h.sync()
    assert torch.equal(out.cpu(), ds.cpu()), "round trip failed"

    # Timed region: K steps, each the encode and the decode of one latent.
    # Step i+1's encode (stream A, handle h) overlaps step i's decode (stream
    # B, a second handle with its own workspace); the inputs rotate over R
    # buffer sets that together exceed L2, so no step finds its data there.
    R = ROTATE_SETS
    hB = codec.Handle(dev)
    hB.check(_abi.fgmm_set_option(hB.ptr, _abi.FGMM_OPT_DECODE_LANES, args.decode_lanes))
    sA, sB = stream, torch.cuda.Stream(dev)
    spA, spB = sptr, ctypes.c_void_p(sB.cuda_stream)
    slot_dp = [dp] + [dp.clone() for _ in range(R - 1)]
    slot_ds = [ds] + [ds.clone() for _ in range(R - 1)]
    slot_desc = [codec.latent(x) for x in slot_dp]
    slot_w = [words] + [torch.empty_like(words) for _ in range(R - 1)]
    slot_o = [offsets] + [torch.empty_like(offsets) for _ in range(R - 1)]
    slot_t = [total] + [torch.empty_like(total) for _ in range(R - 1)]
    slot_out = [out] + [torch.empty_like(out) for _ in range(R - 1)]
    assert sum(x[0].numel() * x[0].element_size() for x in (slot_dp, slot_ds, slot_w, slot_o, slot_out)) == \
        slot_bytes(N, K, S)

    def enc_slot(r):
        h.check(_abi.fgmm_encode(h.ptr, ctypes.byref(slot_desc[r]), slot_ds[r].data_ptr(), S, slot_w[r].data_ptr(),
                                 cap, slot_o[r].data_ptr(), slot_t[r].data_ptr(), spA))

    def dec_slot(r):
        hB.check(_abi.fgmm_decode(hB.ptr, ctypes.byref(slot_desc[r]), slot_w[r].data_ptr(), cap,
                                  slot_o[r].data_ptr(), S, slot_out[r].data_ptr(), spB))

    def run_steps(nsteps, ev=None):
        enc_done = [torch.cuda.Event() for _ in range(nsteps)]
        dec_done = [torch.cuda.Event() for _ in range(nsteps)]
        for i in range(nsteps):
            r = i % R
            if i >= R:
                sA.wait_event(dec_done[i - R])   # slot r's previous decode has read its words
            if ev is not None:
                ev[i][0].record(sA)
            enc_slot(r)
            if ev is not None:
                ev[i][1].record(sA)
            enc_done[i].record(sA)
            sB.wait_event(enc_done[i])
            if ev is not None:
                ev[i][2].record(sB)
            dec_slot(r)
            if ev is not None:
                ev[i][3].record(sB)
            dec_done[i].record(sB)

    run_steps(max(args.warmup, 3))
    torch.cuda.synchronize()
    h.sync(); hB.sync()
    if world > 1:
        dist.barrier()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall0 = time.perf_counter()
    e_start.record(sA)
    sB.wait_event(e_start)
    run_steps(args.steps, ev)
    e_end.record(sB)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    h.sync(); hB.sync()
    for r in range(R):
        assert torch.equal(slot_out[r], ds), "round trip failed in the timed region"
    ms_step = e_start.elapsed_time(e_end) / args.steps
    ms_enc = statistics.mean(ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps))
    ms_dec = statistics.mean(ev[i][2].elapsed_time(ev[i][3]) for i in range(args.steps))
    ms_step, ms_enc, ms_dec = max_over_ranks([ms_step, ms_enc, ms_dec], device=dev)

    # service throughput: D steps decoding at once (step i's decode on
    # stream i mod D, each with its own handle), encode overlapping as above;
    # per-launch decode time grows as the decodes share SMs
    concurrency = {}
    conc_steps = max(R, min(args.steps, 100))
    hD_all = [hB] + [codec.Handle(dev) for _ in range(2)]
    sD_all = [sB] + [torch.cuda.Stream(dev) for _ in range(2)]
    for hx in hD_all[1:]:
        hx.check(_abi.fgmm_set_option(hx.ptr, _abi.FGMM_OPT_DECODE_LANES, args.decode_lanes))
    for D in (2, 3):
        for rep in range(2):   # the first pass grows the new handles' workspaces
            enc_done = [torch.cuda.Event() for _ in range(conc_steps)]
            dec_done = [torch.cuda.Event() for _ in range(conc_steps)]
            dev_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(conc_steps)]
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c0.record(sA)
            for sx in sD_all[:D]:
                sx.wait_event(c0)
            for i in range(conc_steps):
                r, sx, hx = i % R, sD_all[i % D], hD_all[i % D]
                if i >= R:
                    sA.wait_event(dec_done[i - R])
                enc_slot(r)
                enc_done[i].record(sA)
                sx.wait_event(enc_done[i])
                dev_ev[i][0].record(sx)
                hx.check(_abi.fgmm_decode(hx.ptr, ctypes.byref(slot_desc[r]), slot_w[r].data_ptr(), cap,
                                          slot_o[r].data_ptr(), S, slot_out[r].data_ptr(),
                                          ctypes.c_void_p(sx.cuda_stream)))
                dev_ev[i][1].record(sx)
                dec_done[i].record(sx)
            ends = []
            for sx in sD_all[:D]:
                c1 = torch.cuda.Event(enable_timing=True)
                c1.record(sx)
                ends.append(c1)
            torch.cuda.synchronize()
        for hx in [h] + hD_all[:D]:
            hx.sync()
        for r in range(R):
            assert torch.equal(slot_out[r], ds), "round trip failed with concurrent decodes"
        ms_c = max(c0.elapsed_time(c1) for c1 in ends) / conc_steps
        concurrency[str(D)] = {"value": world * N / (ms_c * 1e-3) / 1e6, "ms_per_step": ms_c,
                               "ms_decode_launch": statistics.mean(dev_ev[i][0].elapsed_time(dev_ev[i][1])
                                                                   for i in range(conc_steps))}

    # the same steps one after another on one stream, L2 flushed before each
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ser_steps = max(3, min(args.steps, 50))
    se = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(ser_steps)]
    for i in range(ser_steps):
        flush.fill_(i & 0xff)
        se[i][0].record(stream)
        enc()
        se[i][1].record(stream)
        dec()
        se[i][2].record(stream)
    torch.cuda.synchronize()
    h.sync()
    ser_enc = statistics.mean(se[i][0].elapsed_time(se[i][1]) for i in range(ser_steps))
    ser_dec = statistics.mean(se[i][1].elapsed_time(se[i][2]) for i in range(ser_steps))
    ser_enc, ser_dec = max_over_ranks([ser_enc, ser_dec], device=dev)

    # the table-based comparison coder on the same latent and GPU: builds the
    # per-symbol CDF table (512 entries) and codes from it; same stream
    table = torch.empty((N, 512), dtype=torch.int16, device=dev)
    words_t = torch.empty(cap, dtype=torch.int16, device=dev)
    offsets_t = torch.empty(S // 32 + 1, dtype=torch.int64, device=dev)
    total_t = torch.empty(1, dtype=torch.int64, device=dev)
    out_t = torch.empty(N, dtype=torch.int32, device=dev)

    def tenc():
        h.check(_abi.fgmm_table_encode(h.ptr, L, ds.data_ptr(), S, table.data_ptr(), words_t.data_ptr(), cap,
                                       offsets_t.data_ptr(), total_t.data_ptr(), sptr))

    def tdec():
        h.check(_abi.fgmm_table_decode(h.ptr, L, table.data_ptr(), words.data_ptr(), cap, offsets.data_ptr(), S,
                                       out_t.data_ptr(), sptr))

    tenc(); tdec(); h.sync()
    assert int(total_t.item()) == n_words and torch.equal(words_t[:n_words], words[:n_words]), \
        "table coder stream differs"
    assert torch.equal(out_t, ds), "table decode failed"
    tsteps = max(3, min(args.steps, 20))
    te, td = [], []
    for i in range(tsteps + 2):
        flush.fill_(i & 0xff)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream); tenc(); e1.record(stream); tdec(); e2.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            te.append(e0.elapsed_time(e1)); td.append(e1.elapsed_time(e2))
    h.sync()
    ms_tenc, ms_tdec = statistics.median(te), statistics.median(td)
    del table

    # Sec. V, Table II on this latent: the three approximations of Phi, each
    # coding with its own quantised CDF; time with the lane decoder (the one
    # decoder every approximation runs on), rate against the FP64 mixture
    phi_rows = {}
    words_v = torch.empty(cap, dtype=torch.int16, device=dev)
    off_v = torch.empty(S // 32 + 1, dtype=torch.int64, device=dev)
    tot_v = torch.empty(1, dtype=torch.int64, device=dev)
    out_v = torch.empty(N, dtype=torch.int32, device=dev)
    for name, v in (("a_and_s", _abi.FGMM_PHI_AS), ("logistic", _abi.FGMM_PHI_LOGISTIC),
                    ("polya", _abi.FGMM_PHI_POLYA)):
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_PHI, v))
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 1))

        def venc():
            h.check(_abi.fgmm_encode(h.ptr, L, ds.data_ptr(), S, words_v.data_ptr(), cap, off_v.data_ptr(),
                                     tot_v.data_ptr(), sptr))

        def vdec():
            h.check(_abi.fgmm_decode(h.ptr, L, words_v.data_ptr(), cap, off_v.data_ptr(), S, out_v.data_ptr(), sptr))

        venc(); vdec(); h.sync()
        assert torch.equal(out_v, ds), name
        te_v, td_v = [], []
        for i in range(tsteps + 2):
            flush.fill_(i & 0xff)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream); venc(); e1.record(stream); vdec(); e2.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                te_v.append(e0.elapsed_time(e1)); td_v.append(e1.elapsed_time(e2))
        h.sync()
        aud_v = torch.empty(4, dtype=torch.float64, device=dev)
        h.check(_abi.fgmm_rate_audit(h.ptr, L, ds.data_ptr(), aud_v.data_ptr(), sptr))
        h.sync()
        iv, cv, ev, _ = aud_v.cpu().tolist()
        phi_rows[name] = {"ms_encode": statistics.median(te_v), "ms_decode_lane": statistics.median(td_v),
                          "bits_per_symbol": cv / N, "overhead_pct": 100.0 * (cv / iv - 1.0), "max_cdf_err": ev}
    phi_rows["exact_fp64_bits_per_symbol"] = iv / N
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_PHI, _abi.FGMM_PHI_AS))
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, args.decode_lanes))
    del words_v, off_v, tot_v, out_v

    # rate: FP64 audit on the GPU
    aud = torch.empty(4, dtype=torch.float64, device=dev)
    h.check(_abi.fgmm_rate_audit(h.ptr, L, ds.data_ptr(), aud.data_ptr(), sptr))
    h.sync()
    ideal_bits, coded_bits, max_cdf_err, n_esc = aud.cpu().tolist()

    # end to end through the C ABI from pinned host buffers: H2D parameters
    # and symbols, encode, D2H stream (its length read on the host); H2D
    # stream, decode, D2H symbols. Serial: one step at a time. Pipelined:
    # the same calls with NB buffer sets; input copies, encode, the words'
    # round trip, decode and the symbols' copy back each on a stream of
    # their own, so step i+1's copies and encode overlap step i's decode.
    NB = max(2, args.e2e_buffers)
    hp = torch.from_numpy(lat.params).pin_memory()
    hs = torch.from_numpy(lat.symbols).pin_memory()
    hw = [torch.empty(cap, dtype=torch.int16).pin_memory() for _ in range(NB)]
    ho = [torch.empty(S // 32 + 1, dtype=torch.int64).pin_memory() for _ in range(NB)]
    ht = [torch.empty(1, dtype=torch.int64).pin_memory() for _ in range(NB)]
    hout = [torch.empty(N, dtype=torch.int32).pin_memory() for _ in range(NB)]
    dp2 = [dp] + [torch.empty_like(dp) for _ in range(NB - 1)]
    ds2 = [ds] + [torch.empty_like(ds) for _ in range(NB - 1)]
    desc2 = [codec.latent(x) for x in dp2]
    words2 = [words] + [torch.empty_like(words) for _ in range(NB - 1)]
    off2 = [offsets] + [torch.empty_like(offsets) for _ in range(NB - 1)]
    tot2 = [total] + [torch.empty_like(total) for _ in range(NB - 1)]
    dwords2 = [torch.empty(cap, dtype=torch.int16, device=dev) for _ in range(NB)]
    doff2 = [torch.empty(S // 32 + 1, dtype=torch.int64, device=dev) for _ in range(NB)]
    out2 = [out] + [torch.empty_like(out) for _ in range(NB - 1)]
    cs = stream
    xs = torch.cuda.Stream(dev)    # host-to-device inputs
    ys = torch.cuda.Stream(dev)    # words round trip
    zs = torch.cuda.Stream(dev)    # decoded symbols back to the host
    csp = ctypes.c_void_p(cs.cuda_stream)
    dcs = sB                       # decode: its own stream and handle, overlapping the next step's encode
    dcsp = ctypes.c_void_p(dcs.cuda_stream)
    ev_in, ev_enc, ev_words, ev_dec, ev_free = ([torch.cuda.Event() for _ in range(NB)] for _ in range(5))
    nw_last = [0] * NB

    def issue_inputs(i, xst):
        b = i % NB
        with torch.cuda.stream(xst):
            if i >= NB:
                xst.wait_event(ev_free[b])
            dp2[b].copy_(hp, non_blocking=True)
            ds2[b].copy_(hs, non_blocking=True)
            ev_in[b].record(xst)

    def issue_encode(i):
        b = i % NB
        cs.wait_event(ev_in[b])
        h.check(_abi.fgmm_encode(h.ptr, ctypes.byref(desc2[b]), ds2[b].data_ptr(), S, words2[b].data_ptr(), cap,
                                 off2[b].data_ptr(), tot2[b].data_ptr(), csp))
        with torch.cuda.stream(cs):
            ht[b].copy_(tot2[b], non_blocking=True)
            ho[b].copy_(off2[b], non_blocking=True)
        ev_enc[b].record(cs)

    def finish(i, yst, zst):
        b = i % NB
        ev_enc[b].synchronize()
        nw = int(ht[b].item())
        nw_last[b] = nw
        with torch.cuda.stream(yst):
            yst.wait_event(ev_enc[b])
            hw[b][:nw].copy_(words2[b][:nw], non_blocking=True)
            dwords2[b][:nw].copy_(hw[b][:nw], non_blocking=True)
            doff2[b].copy_(ho[b], non_blocking=True)
            ev_words[b].record(yst)
        dcs.wait_event(ev_words[b])
        hB.check(_abi.fgmm_decode(hB.ptr, ctypes.byref(desc2[b]), dwords2[b].data_ptr(), nw, doff2[b].data_ptr(), S,
                                  out2[b].data_ptr(), dcsp))
        ev_dec[b].record(dcs)
        with torch.cuda.stream(zst):
            zst.wait_event(ev_dec[b])
            hout[b].copy_(out2[b], non_blocking=True)
            ev_free[b].record(zst)

    # serial: every step waits for the previous one (one stream, one buffer set)
    e2e_t = []
    for i in range(args.e2e_steps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        issue_inputs(0, cs)
        issue_encode(0)
        finish(0, cs, cs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if i >= 2:
            e2e_t.append(dt)
    h.sync(); hB.sync()
    assert torch.equal(hout[0], hs), "end-to-end round trip failed"
    e2e_serial_ms = 1e3 * statistics.median(e2e_t)
    # pipelined: step i+1's inputs and encode are issued before step i's decode
    n_pipe = max(args.e2e_steps, 2 * NB)
    for rep in range(2):   # the first pass warms the second stream and the buffers
        for x in hout:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        issue_inputs(0, xs)
        issue_encode(0)
        for i in range(n_pipe):
            if i + 1 < n_pipe:
                issue_inputs(i + 1, xs)
                issue_encode(i + 1)
            finish(i, ys, zs)
        torch.cuda.synchronize()
        e2e_ms = 1e3 * (time.perf_counter() - t0) / n_pipe
    h.sync(); hB.sync()
    assert all(torch.equal(x, hs) for x in hout), "pipelined end-to-end round trip failed"
    nw = nw_last[0]
    h2d = hp.numel() * 4 + hs.numel() * 4 + nw * 2 + ho[0].numel() * 8
    d2h = 8 + ho[0].numel() * 8 + nw * 2 + hout[0].numel() * 4
    e2e_ms, e2e_serial_ms = max_over_ranks([e2e_ms, e2e_serial_ms], device=dev)

    value = world * N / (ms_step * 1e-3) / 1e6
    plan = codec.decode_plan(S, h=h)
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_derived = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12   # Tops/s
    alu_peak = alu_peaks["fma"]
    ops = cdf_evals * ops_per_eval(K)
    achieved = ops / (ms_dec * 1e-3) / 1e12
    result = {
        "metric": "encode+decode Msymbols/s (round trip)",
        "value": value,
        "unit": "Msymbols/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(args.warmup, 3),
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(N, K, S),
        "schedule": "step i+1's encode overlaps step i's decode on a second stream (own handle)",
        "concurrent_decodes": concurrency,
        "serial": {"value": world * N / ((ser_enc + ser_dec) * 1e-3) / 1e6, "ms_per_step": ser_enc + ser_dec,
                   "ms_encode": ser_enc, "ms_decode": ser_dec,
                   "l2": "flushed before each step (256 MiB write outside the timed events)"},
        "encode_msym_s": world * N / (ms_enc * 1e-3) / 1e6,
        "decode_msym_s": world * N / (ms_dec * 1e-3) / 1e6,
        "ms_encode": ms_enc,
        "ms_decode": ms_dec,
        "bits_per_symbol": 16.0 * n_words / N,
        "cdf_evals_per_symbol": cdf_evals / max(nsym, 1),
        "decode_lanes": args.decode_lanes or "auto",
        "table_coder": {"encode_msym_s": N / (ms_tenc * 1e-3) / 1e6, "decode_msym_s": N / (ms_tdec * 1e-3) / 1e6,
                        "ms_encode": ms_tenc, "ms_decode": ms_tdec, "table_mb": N * 512 * 2 / 1e6,
                        "encode_speedup_table_free": ms_tenc / ser_enc, "decode_speedup_table_free": ms_tdec / ser_dec,
                        "stream_identical": True},
        "phi_approximations": phi_rows,
        "rate": {"ideal_bits_per_symbol": ideal_bits / N, "coded_bits_per_symbol": coded_bits / N,
                 "overhead_pct": 100.0 * (coded_bits / ideal_bits - 1.0),
                 "container_overhead_pct": 100.0 * (16.0 * n_words / coded_bits - 1.0),
                 "max_cdf_err": max_cdf_err, "escapes": int(n_esc), "audit": "FP64 on the GPU (erfc)"},
        "gpu_launches": launches_per_step * args.steps,
        "wall_s_timed_region": t_wall,
        "e2e": {"value": world * N / (e2e_ms * 1e-3) / 1e6, "unit": "Msymbols/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "pipeline_buffers": NB,
                "serial_value": world * N / (e2e_serial_ms * 1e-3) / 1e6},
        "roofline": {"kernel": plan["kernel"], "lanes": plan["lanes"], "cluster": plan["cluster"],
                     "round0": plan["round0"],
                     "bound": "alu", "achieved": achieved, "peak": alu_peak,
                     "unit": "Tops/s (FP32 lane ops)", "frac": achieved / alu_peak,
                     "traffic": DECODE_TRAFFIC_BYTES.get(f'{plan["kernel"]}/{plan["lanes"]}/{plan["cluster"]}/{plan["round0"]}'),
                     "peak_source": "measured: FP32 FMA chains on every SM (fgmm_peak_probe), CUDA events",
                     "peak_derived": alu_derived,
                     "peak_derived_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                            f"{sm_max:.0f} MHz",
                     "xu_peak": alu_peaks["rcp"],
                     "xu_peak_source": "measured: rcp.approx chains on every SM (fgmm_peak_probe)",
                     "ops_per_cdf_eval": ops_per_eval(K),
                     "ops_count": f"{OPS_PER_PHI} FP32 operations per Phi-hat x K components per CDF evaluation",
                     # the decode is a chain of dependent steps per stream:
                     # its time per step at the sampled SM clock
                     "steps_per_stream": -(-N // S),
                     "cycles_per_step": ms_dec * 1e-3 * (clk["sm_mhz"] if clk else sm_max) * 1e6 / -(-N // S)},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(lat, S)
    if not args.no_throughput:
        result["throughput"] = throughput_workloads(dev, alu_peak, float(peaks.get("hbm_gbs", 6800.0)))
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def run_batch_only(args):
    import torch
    from paper_2509_18815_gb300 import build, codec, synth
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = codec.handle(dev)
    peaks = measured_peaks()
    alu_peak = measure_alu_peaks(dev, h)["fma"]
    shapes = synth.batch_shapes(64, seed=1004)[: args.batch_only]
    out = {}
    batch_case(dev, h, out, f"batch{len(shapes)}_uneven_k3",
               [synth.make_latent(C, H, W, 3, 1004 + i) for i, (C, H, W) in enumerate(shapes)], alu_peak,
               float(peaks.get("hbm_gbs", 6800.0)), reps=max(args.steps, 1), max_overhead=args.batch_overhead,
               table=args.batch_table)
    print(json.dumps(out))


def run_gsm_only(args):
    import torch
    from paper_2509_18815_gb300 import build, codec
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = codec.handle(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    print(json.dumps({"gsm_320x64x96": gsm_case(dev, h, flush, max(args.steps, 1))}))


def run_proposal_only(args):
    import torch
    from paper_2509_18815_gb300 import build, codec
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = codec.handle(dev)
    alu_peak = measure_alu_peaks(dev, h)["fma"]
    res = proposal_case(dev, h, alu_peak, reps=max(args.steps, 1), n_latents=args.proposal_latents,
                        train_scale=args.proposal_train_scale)
    print(json.dumps({f"proposal_{args.proposal_latents}x320x64x96_sigma64": res}))


def run_ckbd_only(args):
    """The checkerboard two-pass case alone. Its first decoder launch is the
    fused two-pass decode of fgmm_ckbd_decode."""
    import torch
    from paper_2509_18815_gb300 import build, codec
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = codec.handle(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    print(json.dumps({"ckbd_192x32x48_k3": ckbd_case(dev, h, flush, max(args.steps, 1))}))


def run_traffic_probe(args):
    """Each kernel that has a roofline line in the benchmark, launched once
    after one warm-up, for an ncu capture of DRAM bytes per launch: the
    192x32x48 latent at 1024 streams (interval, rANS encode, scan,
    compaction; decoder), the 320x64x96 K = 3 latent at the autotuned stream
    count (the same kernels), the first 8 latents of the 64-latent batch
    (batch encode, scan, compaction; batch decode), and 2 latents of
    320x64x96 with scales up to 64 through the batched proposal decoder (a
    zero network). Prints the symbols each case codes."""
    import torch
    from paper_2509_18815_gb300 import build, codec, synth
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = codec.handle(dev)
    cases = {}
    for name, (C, H, W, seed, S) in {"latent_192x32x48": (192, 32, 48, 1002, 1024),
                                     "latent_320x64x96": (320, 64, 96, 1003, None)}.items():
        lat = synth.make_latent(C, H, W, 3, seed)
        dp = torch.from_numpy(lat.params).to(dev)
        ds = torch.from_numpy(lat.symbols).to(dev)
        S = S or codec.autotune([lat.N], h=h)[0]
        for _ in range(2):   # warm-up, then the captured launches
            words, off = codec.encode(dp, ds, S, h=h)
            codec.decode(dp, words, off, S, h=h)
        cases[name] = {"symbols": lat.N, "S": S, "decoder": codec.decode_plan(S, h=h)["kernel"]}
    shapes = synth.batch_shapes(64, seed=1004)[:8]
    lats = [synth.make_latent(C, H, W, 3, 1004 + i) for i, (C, H, W) in enumerate(shapes)]
    b = codec.Batch([torch.from_numpy(l.params).to(dev) for l in lats],
                    [torch.from_numpy(l.symbols).to(dev) for l in lats], h=h)
    for _ in range(2):
        b.encode()
        b.decode()
    cases["batch8"] = {"symbols": sum(l.N for l in lats), "segments": b.seg_base[-1]}
    b.close()
    lats = [synth.make_latent(320, 64, 96, 3, seed=1105 + i, sigma_max=64.0) for i in range(2)]
    b = codec.Batch([torch.from_numpy(l.params).to(dev) for l in lats],
                    [torch.from_numpy(l.symbols).to(dev) for l in lats], h=h)
    b.encode()
    P = codec.mlp_pack(torch.zeros(_mlp_params(), dtype=torch.float32, device=dev), h=h)
    for _ in range(2):
        b.decode_proposal(P)
    cases["proposal2_sigma64"] = {"symbols": sum(l.N for l in lats), "segments": b.seg_base[-1]}
    b.close()
    print(json.dumps({"traffic_probe": cases}))


def _mlp_params():
    from paper_2509_18815_gb300 import _abi
    return _abi.FGMM_MLP_PARAMS


def main():
    args = parse()
    if args.batch_only > 0:
        run_batch_only(args)
    elif args.gsm_only:
        run_gsm_only(args)
    elif args.proposal_only:
        run_proposal_only(args)
    elif args.ckbd_only:
        run_ckbd_only(args)
    elif args.traffic_probe:
        run_traffic_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_fgmm(args)


if __name__ == "__main__":
    main()
