"""Autotuner for libsu3's launch configurations.

For each form (dtype x repr x layout) it times su3_mult over a grid of launch configurations
(block, tile_sites, stages, ctas_per_sm and, for AOS, threads per link: one per link or one per
output row) on a lattice larger than L2, with CUDA events after
warm-up, and keeps the fastest. The batched kernel's tile/block/stages are tuned the same way on
the 96-lattice batch. Results go to ``tune_cache.json`` beside this file, keyed by GPU name and SM
count, and ``apply_cached`` installs them on a handle (bench.py and the tests use the same).

    python -m paper_2103_00571_gb300.tune [--L 48] [--forms all|f64-full-aos-f32pair,...] [--batched]
    python -m paper_2103_00571_gb300.tune --time-batched 5 [--arith f32pair]   # time the batch only

Form names are dtype-repr-layout[-arith][-p<stride>], e.g. f16-2row-aosoa32 or
f64-full-aos-f32pair-p640 (the paper's padded 640-byte FP64 site); repr is full (FULL18 in and
out), 2row (TWOROW12 in and out) or 2to18 (TWOROW12 in, FULL18 out: its own launch shape, set
with su3_set_launch_cfg_for). ``best_layout`` ranks the tuned layouts of a storage type, and
``apply_cached`` installs the configurations on a handle.
"""
import argparse
import itertools
import json
import os
import time

import numpy as np

from . import _binding as B

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")

DT = {"f64": B.F64, "f32": B.F32, "f16": B.F16, "bf16": B.BF16}
RP = {"full": B.FULL18, "2row": B.TWOROW12}
LY = {"aos": B.AOS, "aosoa32": B.AOSOA32, "soa": B.SOA}
AR = {"native": B.NATIVE, "f32pair": B.F32PAIR, "hybrid": B.HYBRID}


def form_name(desc):
    """dtype-repr-layout-arith, plus -p<stride> for a padded AOS site (e.g. the paper's 640 B)."""
    inv = lambda m, v: [k for k, x in m.items() if x == v][0]  # noqa: E731
    name = "%s-%s-%s-%s" % (inv(DT, desc.dtype), inv(RP, desc.repr), inv(LY, desc.layout), inv(AR, desc.arith))
    packed = 4 * B.link_bytes(desc.dtype, desc.repr)
    if desc.layout == B.AOS and desc.site_stride_bytes not in (0, packed):
        name += "-p%d" % desc.site_stride_bytes
    return name


def parse_pair(name, n_sites=0):
    """(a form, c form) of a form name; the two differ only for 2to18 (two-row in, full out)."""
    parts = name.split("-")
    stride = 0
    if parts[-1].startswith("p") and parts[-1][1:].isdigit():
        stride = int(parts.pop()[1:])
    d, r, l, a = (parts + ["native"])[:4]
    r_in, r_out = (B.TWOROW12, B.FULL18) if r == "2to18" else (RP[r], RP[r])
    return (B.Desc(DT[d], r_in, LY[l], n_sites, stride, AR[a]), B.Desc(DT[d], r_out, LY[l], n_sites, stride, AR[a]))


def parse_form(name, n_sites=0):
    return parse_pair(name, n_sites)[0]


def is_pair_name(name):
    return "-2to18-" in name


# The default grid. HYBRID forms (f64-*-hybrid) can still be named with --forms; they are left out
# here because they measured slower than pure F32PAIR in every configuration tried.
ALL_FORMS = ["f64-full-aos-f32pair", "f64-2to18-aos-f32pair", "f64-2to18-aos",
             "f64-full-aosoa32-f32pair", "f64-2row-aos-f32pair", "f64-full-aos", "f32-full-aos", "f16-full-aos", "bf16-full-aos", "f64-2row-aos", "f32-2row-aos",
             "f16-2row-aos", "f64-full-soa", "f32-full-soa", "f16-full-soa", "f64-full-aosoa32",
             "f32-full-aosoa32", "f16-full-aosoa32", "bf16-full-aosoa32",
             "f64-full-aos-native-p640", "f64-full-aos-f32pair-p640"]


def gpu_key():
    import torch
    p = torch.cuda.get_device_properties(0)
    return "%s/%d" % (p.name, p.multi_processor_count)


def load_cache():
    if not os.path.exists(CACHE):
        return {}
    with open(CACHE) as f:
        return json.load(f)


def apply_cached(h, key=None):
    """Installs the cached configurations for this GPU on handle ``h``; returns what it applied."""
    cache = load_cache()
    key = key or gpu_key()
    entry = cache.get(key, {})
    for name, cfg in entry.get("forms", {}).items():
        if is_pair_name(name):
            h.set_launch_cfg_for(*parse_pair(name), **cfg["cfg"])
        else:
            h.set_launch_cfg(parse_form(name), **cfg["cfg"])
    if "batched" in entry:
        h.set_batched_cfg(**entry["batched"]["cfg"])
    return entry


def best_layout(dtype, repr_=None, arith=None, key=None):
    """The internal layout (AOS, AOSOA32 or SOA) with the highest tuned GB/s for this storage type,
    representation and arithmetic on this GPU, from the tuning cache; None if none was tuned.
    (Data arrives as AOS, the benchmark's format; pack once into the winner to reuse it.)"""
    repr_ = B.FULL18 if repr_ is None else repr_
    arith = B.NATIVE if arith is None else arith
    if key is None:
        key = gpu_key()
    forms = load_cache().get(key, {}).get("forms", {})
    best = None
    for name, rec in forms.items():
        if is_pair_name(name):
            continue
        d = parse_form(name)
        if d.site_stride_bytes:  # padded AOS sites are a storage format, not a layout choice
            continue
        if (d.dtype, d.repr, d.arith) == (dtype, repr_, arith) and (best is None or rec["GBps"] > best[0]):
            best = (rec["GBps"], d.layout)
    return None if best is None else best[1]


def candidates(desc, out=None):
    """Launch configurations to time for form `desc` (a), writing form `out` (c; default: desc)."""
    out = desc if out is None else out
    if desc.arith == B.HYBRID:
        # one or two native warps per CTA; AOS tiles hold at least one link per thread
        out = []
        for c in candidates(B.Desc(desc.dtype, desc.repr, desc.layout, desc.n_sites, 0, B.F32PAIR)):
            warps = c["block"] // 32
            if desc.layout == B.AOS and c["tile_sites"] * 4 < c["block"]:
                continue
            out += [dict(c, native_permille=nw * 1000 // warps) for nw in (1, 2) if nw < warps]
        return out
    rows = 3 if out.repr == B.FULL18 else 2  # output rows: threads per link under the row split
    if desc.layout == B.AOS:
        site = B.link_bytes(desc.dtype, desc.repr) * 4  # shared-memory tiles are packed whatever the stride
        out = []  # threads_per_link 3 = one thread per output row
        for block, stages, cps, tpl in itertools.product((64, 128, 192, 256), (3, 4, 6), (1, 2, 3), (1, 3)):
            # tiles of ~9/18/36 KB, and tiles of exactly one or two links per thread
            sizes = sorted({max(8, tb // site) for tb in (9216, 18432, 36864)} | {block // 4, block // 2})
            for ts in sizes:
                smem = 1024 + stages * ((ts * site + 127) // 128 * 128)
                if smem > 227 * 1024 or (smem + 1024) * cps > 228 * 1024 or 4 * ts * (rows if tpl == 3 else 1) < block:
                    continue
                out.append(dict(block=block, tile_sites=ts, stages=stages, ctas_per_sm=cps, threads_per_link=tpl))
        return out
    # element-major layouts: direct global loads (stages 0: tile_sites = links per thread) ...
    out = [dict(block=bl, tile_sites=lpt, ctas_per_sm=c) for bl in (128, 256) for lpt in (1, 2, 4)
           for c in (2, 4, 8)]
    # ... or the staged kernel (AOSOA32 tiles of whole 32-link blocks; SOA tiles of <= 64 sites in
    # element planes of 256 links, so an SOA stage is the same size whatever the tile)
    link = B.link_bytes(desc.dtype, desc.repr)
    for block, stages, cps, tpl in itertools.product((64, 128, 192, 256), (2, 3, 4, 6), (1, 2, 3, 4), (1, 3)):
        if desc.layout == B.SOA:
            sizes = {64, 32}
        else:
            sizes = {max(8, tb // (4 * link) // 8 * 8) for tb in (9216, 18432, 36864)} | {max(8, block // 4 // 8 * 8)}
        for ts in sorted(sizes):
            stage = link * 4 * (64 if desc.layout == B.SOA else ts)
            smem = 1024 + stages * ((stage + 127) // 128 * 128)
            if smem > 227 * 1024 or (smem + 1024) * cps > 228 * 1024 or 4 * ts * (rows if tpl == 3 else 1) < block:
                continue
            out.append(dict(block=block, tile_sites=ts, stages=stages, ctas_per_sm=cps, threads_per_link=tpl))
    return out


def time_cfg(h, desc, abuf, b, cbuf, cfg, reps=5, iters=4, out=None):
    import torch
    out = desc if out is None else out
    if out.repr != desc.repr:
        h.set_launch_cfg_for(desc, out, **cfg)
    else:
        h.set_launch_cfg(desc, **cfg)
    s = torch.cuda.current_stream()
    for _ in range(2):
        h.mult(desc, abuf, b, out, cbuf)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(iters):
            h.mult(desc, abuf, b, out, cbuf)
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / iters)
    h.sync()
    return float(np.median(ts))


def tune_forms(h, names, L=48, log=print):
    import torch

    import su3_inputs as gen
    V = L ** 4
    a64 = torch.from_numpy(gen.sites(gen.DEFAULT_SEED, 0, V)).cuda()
    b = gen.bmat(gen.DEFAULT_SEED, 0, V)
    results = {}
    for name in names:
        d, dc = parse_pair(name, V)
        abuf = torch.empty(B.array_bytes(d), dtype=torch.uint8, device="cuda")
        cbuf = torch.empty(B.array_bytes(dc), dtype=torch.uint8, device="cuda")
        h.pack(a64, d, abuf)
        best = None
        for cfg in candidates(d, dc):
            ms = time_cfg(h, d, abuf, b, cbuf, cfg, out=dc)
            if best is None or ms < best[0]:
                best = (ms, cfg)
        gbs = ((B.link_bytes(d.dtype, d.repr) + B.link_bytes(dc.dtype, dc.repr)) * 4 * V) / (best[0] * 1e-3) / 1e9
        results[name] = {"cfg": best[1], "ms": round(best[0], 4), "GBps": round(gbs, 1), "L": L}
        log("%-22s %s  %.3f ms  %.0f GB/s" % (name, best[1], best[0], gbs))
        del abuf, cbuf
    return results


def make_batch96(h, arith=None):
    """The 96-lattice workload: extents drawn from {4, 6, ..., 24}, FP64 (even index) / FP32 (odd),
    each lattice with its own b. FP64 lattices take ``arith`` (default NATIVE). Returns the batch
    items and the device buffers that must stay alive while they are used."""
    import ctypes

    import torch

    import su3_inputs as gen
    arith = B.NATIVE if arith is None else arith
    ext = gen.extents(gen.DEFAULT_SEED, 96)
    items, keep = [], []
    for k in range(96):
        V = int(np.prod(ext[k]))
        dt = B.F64 if k % 2 == 0 else B.F32
        d = B.Desc(dt, B.FULL18, B.AOS, V, 0, arith if dt == B.F64 else B.NATIVE)
        a = torch.from_numpy(gen.sites(gen.DEFAULT_SEED, k, V)).cuda()
        abuf = torch.empty(B.array_bytes(d), dtype=torch.uint8, device="cuda")
        h.pack(a, d, abuf)
        cbuf = torch.empty_like(abuf)
        keep += [abuf, cbuf]
        items.append(B.BatchItem(d, abuf.data_ptr(), cbuf.data_ptr(),
                                 (ctypes.c_double * 72)(*gen.bmat(gen.DEFAULT_SEED, k, V))))
    h.sync()
    return items, keep


def time_batched(h, items, reps=10, warm=3):
    """Mean ms of one graph-replayed batched launch (CUDA events on the current stream)."""
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warm):
        h.mult_batched(items, s, use_graph=True)
    h.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        h.mult_batched(items, s, use_graph=True)
    e1.record(s)
    e1.synchronize()
    h.sync()
    return e0.elapsed_time(e1) / reps


def tune_batched(h, log=print):
    items, keep = make_batch96(h)
    best = None
    for block, ts, stages, cps, tpl in itertools.product((64, 128, 256), (16, 32, 64), (2, 3, 4), (1, 2, 3, 4, 6),
                                                         (1, 3)):
        if 1024 + stages * ((ts * 576 + 127) // 128 * 128) > 227 * 1024 // cps or block * cps > 1024:
            continue
        cfg = dict(block=block, tile_sites=ts, stages=stages, ctas_per_sm=cps, threads_per_link=tpl)
        h.set_batched_cfg(**cfg)
        ms = time_batched(h, items)
        if best is None or ms < best[0]:
            best = (ms, cfg)
    h.set_batched_cfg(**best[1])
    log("batched %s %.3f ms" % (best[1], best[0]))
    return {"cfg": best[1], "ms": round(best[0], 4)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=48)
    ap.add_argument("--forms", default="all")
    ap.add_argument("--batched", action="store_true")
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--time-batched", type=int, default=0, metavar="REPS",
                    help="only time the 96-lattice batch under the cached configuration (REPS graph replays)")
    ap.add_argument("--arith", default="native", choices=["native", "f32pair"],
                    help="arithmetic of the FP64 lattices for --time-batched")
    args = ap.parse_args()
    h = B.Handle(0)
    if args.time_batched:
        apply_cached(h)
        items, keep = make_batch96(h, AR[args.arith])
        ms = time_batched(h, items, reps=args.time_batched)
        sites = sum(it.desc.n_sites for it in items)
        print(json.dumps({"workload": "96-lattice batch", "arith": args.arith, "ms": round(ms, 4),
                          "site_updates_per_s": round(sites / (ms * 1e-3), 1), "cfg": h.get_batched_cfg()}))
        return
    names = ALL_FORMS if args.forms == "all" else args.forms.split(",")
    cache = load_cache()
    key = gpu_key()
    entry = cache.get(key, {"forms": {}})
    t0 = time.time()
    entry["forms"].update(tune_forms(h, names, args.L))
    if args.batched:
        entry["batched"] = tune_batched(h)
    entry["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    cache[key] = entry
    with open(args.out, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    print("tuned %d forms in %.0f s -> %s" % (len(names), time.time() - t0, args.out))


if __name__ == "__main__":
    main()
