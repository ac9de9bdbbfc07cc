"""Summaries of ncu CSV captures for the committed profiles.

    python -m paper_1311_1695_gb300.profile_summary launches CAPTURE.csv
        per kernel: launches, total device time, share (markdown table);
    python -m paper_1311_1695_gb300.profile_summary metrics CAPTURE.csv
        per kernel: the mean of every captured metric (markdown table);
    python -m paper_1311_1695_gb300.profile_summary traffic CAPTURE.csv --key pcg_split@c5 \\
            --model-bytes B --sources pcg_split.cu spmm.cu [--regex R]
        the DRAM bytes (read + write) of the captured launches over the
        algorithmic bytes B of the same launches, written into
        profiles/traffic.json under the key with the sources' digest (bench.py
        scales the ratio by each launch's algorithmic bytes and reports null
        once a source changed).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
from collections import defaultdict

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rows(path):
    data = list(csv.reader(open(path)))
    for i, r in enumerate(data):
        if r and r[0] == "ID":
            hdr = data[i]
            return [dict(zip(hdr, r)) for r in data[i + 1:] if len(r) >= len(hdr)]
    return []


def short(name: str) -> str:
    n = name.split("(")[0].replace("void ", "")
    return n.split("::")[-1]


def to_us(v: float, unit: str) -> float:
    return {"ns": v / 1e3, "nsecond": v / 1e3, "usecond": v, "us": v, "msecond": v * 1e3, "ms": v * 1e3}.get(unit, v / 1e3)


def launches(path):
    agg = defaultdict(lambda: [0, 0.0])
    for x in rows(path):
        if x["Metric Name"] != "gpu__time_duration.sum":
            continue
        a = agg[short(x["Kernel Name"])]
        a[0] += 1
        a[1] += to_us(float(x["Metric Value"].replace(",", "")), x.get("Metric Unit", "ns"))
    tot = sum(v[1] for v in agg.values()) or 1.0
    out = ["| kernel | launches | total (us) | share |", "|---|---|---|---|"]
    for k, (n, us) in sorted(agg.items(), key=lambda t: -t[1][1]):
        out.append(f"| `{k}` | {n} | {us:.1f} | {100 * us / tot:.1f} % |")
    out.append(f"| total | {sum(v[0] for v in agg.values())} | {tot:.1f} | |")
    return "\n".join(out)


def metrics(path):
    agg = defaultdict(lambda: defaultdict(list))
    units = {}
    for x in rows(path):
        agg[short(x["Kernel Name"])][x["Metric Name"]].append(float(x["Metric Value"].replace(",", "")))
        units[x["Metric Name"]] = x.get("Metric Unit", "")
    out = []
    for k, mm in agg.items():
        out.append(f"### `{k}` ({len(next(iter(mm.values())))} launches)\n")
        out.append("| metric | mean | unit |\n|---|---|---|")
        for m, v in sorted(mm.items()):
            out.append(f"| {m} | {sum(v) / len(v):.4g} | {units.get(m, '')} |")
        out.append("")
    return "\n".join(out)


def traffic(path, key, model_bytes, sources, regex=None):
    tot = 0.0
    n = 0
    for x in rows(path):
        if x["Metric Name"] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        if regex and not re.search(regex, x["Kernel Name"]):
            continue
        v = float(x["Metric Value"].replace(",", ""))
        u = x.get("Metric Unit", "byte")
        tot += v * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(u, 1)
        n += 1
    h = hashlib.sha256()
    for s in sources:
        h.update(open(os.path.join(ROOT, "paper_1311_1695_gb300", "csrc", s), "rb").read())
    p = os.path.join(ROOT, "profiles", "traffic.json")
    d = json.load(open(p)) if os.path.exists(p) else {}
    d[key] = {"sources": list(sources), "source_sha": h.hexdigest()[:16], "dram_bytes": round(tot),
              "model_bytes": round(model_bytes), "dram_over_model": round(tot / model_bytes, 4),
              "metric_rows": n}
    json.dump(d, open(p, "w"), indent=1)
    return d[key]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["launches", "metrics", "traffic"])
    ap.add_argument("csv")
    ap.add_argument("--key")
    ap.add_argument("--model-bytes", type=float)
    ap.add_argument("--sources", nargs="*", default=[])
    ap.add_argument("--regex")
    a = ap.parse_args(argv)
    if a.what == "launches":
        print(launches(a.csv))
    elif a.what == "metrics":
        print(metrics(a.csv))
    else:
        print(json.dumps(traffic(a.csv, a.key, a.model_bytes, a.sources, a.regex), indent=1))


if __name__ == "__main__":
    main()
