"""Summarise an ncu launch list (``--metrics gpu__time_duration.sum --csv``)
into per-kernel launches, total time and share of the captured GPU time.

    python -m paper_2606_13825_b300.ncu_summary launches.csv
"""
import csv
import re
import sys
from collections import defaultdict


def summarise(path):
    rows = list(csv.reader(open(path)))
    hdr = None
    for i, r in enumerate(rows):
        if "Kernel Name" in r and "Metric Value" in r:
            hdr = i
            break
    if hdr is None:
        raise ValueError("no ncu CSV header found")
    h = rows[hdr]
    ki, mi, vi, ui = h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit")
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for r in rows[hdr + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r[ki]).replace("void ", "").strip()
        name = re.sub(r"<.*", "", name)
        scale = {"nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "second": 1e3}.get(r[ui], 1e-6)
        tot[name] += float(r[vi].replace(",", "")) * scale
        cnt[name] += 1
    all_ms = sum(tot.values())
    out = []
    for k in sorted(tot, key=lambda k: -tot[k]):
        out.append((k, cnt[k], tot[k], tot[k] / all_ms))
    return out, all_ms


if __name__ == "__main__":
    res, all_ms = summarise(sys.argv[1])
    print(f"{'kernel':40s} {'launches':>9s} {'total ms':>11s} {'share':>7s}")
    for k, n, ms, sh in res:
        print(f"{k:40s} {n:9d} {ms:11.3f} {100 * sh:6.2f}%")
    print(f"{'all':40s} {sum(r[1] for r in res):9d} {all_ms:11.3f}")
