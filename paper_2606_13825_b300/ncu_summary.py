"""Summaries of ncu output for the committed profile notes.

Launch list (``ncu --metrics gpu__time_duration.sum --csv``): launches, total
time and share of the captured GPU time per kernel.

    python -m paper_2606_13825_b300.ncu_summary launches.csv

One capture exported with ``ncu -i report.ncu-rep --page raw --csv``: the
metrics the roofline and stall analysis use, as a markdown table.

    python -m paper_2606_13825_b300.ncu_summary --raw report_raw.csv
"""
import csv
import re
import sys
from collections import defaultdict

_TIME_TO_MS = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
               "s": 1e3, "second": 1e3}

RAW_METRICS = [
    ("gpu__time_duration.sum", "duration"),
    ("dram__bytes_read.sum", "DRAM read"),
    ("dram__bytes_write.sum", "DRAM write"),
    ("gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed", "DRAM throughput % of peak"),
    ("sm__throughput.avg.pct_of_peak_sustained_elapsed", "SM throughput % of peak"),
    ("smsp__issue_active.avg.pct_of_peak_sustained_active", "issue slots busy %"),
    ("sm__warps_active.avg.pct_of_peak_sustained_active", "warps active % of max"),
    ("launch__grid_size", "grid"),
    ("launch__block_size", "block"),
    ("launch__registers_per_thread", "registers / thread"),
    ("launch__occupancy_limit_shared_mem", "CTAs / SM (shared-memory limit)"),
    ("smsp__inst_executed.sum", "warp instructions"),
    ("l1tex__data_pipe_lsu_wavefronts_mem_shared.sum", "shared-memory wavefronts"),
    ("l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum", "shared-memory bank conflicts"),
    ("l1tex__data_pipe_tc_wavefronts_mem_shared.sum", "tensor-core shared-memory wavefronts"),
    ("TPC.TriageCompute.sm__pipe_tensor_subpipe_hmma_cycles_active_realtime.avg", "tensor pipe (HMMA) active cycles / SM"),
    ("TPC.TriageCompute.sm__pipe_tensor_cycles_active_realtime.avg.pct_of_peak_sustained_elapsed", "tensor pipe active % of elapsed"),
    ("sm__inst_executed_pipe_tc.avg.pct_of_peak_sustained_active", "tensor-core instructions % of peak"),
    ("sm__cycles_active.avg", "SM active cycles (mean)"),
    ("sm__cycles_active.max", "SM active cycles (max)"),
    ("gpc__cycles_elapsed.max", "elapsed cycles"),
]


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
        tot[name] += float(r[vi].replace(",", "")) * _TIME_TO_MS.get(r[ui], 1e-6)
        cnt[name] += 1
    all_ms = sum(tot.values())
    out = []
    for k in sorted(tot, key=lambda k: -tot[k]):
        out.append((k, cnt[k], tot[k], tot[k] / all_ms))
    return out, all_ms


def raw_table(path):
    """Markdown rows (kernel, metric, value unit) of one raw-page export;
    the second CSV row holds the units."""
    rows = list(csv.reader(open(path)))
    hdr, units = rows[0], rows[1]
    lines = []
    for r in rows[2:]:
        name = r[hdr.index("Kernel Name")]
        lines.append(f"**{name[:100]}**\n")
        lines.append("| metric | value |")
        lines.append("|---|---|")
        for key, label in RAW_METRICS:
            if key in hdr:
                i = hdr.index(key)
                lines.append(f"| {label} (`{key}`) | {r[i]} {units[i]} |")
        stalls = []
        for i, k in enumerate(hdr):
            if k.startswith("smsp__average_warps_issue_stalled_") and k.endswith("_per_issue_active.ratio"):
                try:
                    stalls.append((float(r[i]), k[len("smsp__average_warps_issue_stalled_"):-len("_per_issue_active.ratio")]))
                except ValueError:
                    pass
        stalls.sort(reverse=True)
        lines.append("| top warp stalls (cycles per issue) | " +
                     ", ".join(f"{n} {v:.2f}" for v, n in stalls[:6]) + " |")
        lines.append("")
    return "\n".join(lines)


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[1] == "--raw":
        print(raw_table(sys.argv[2]))
    else:
        res, all_ms = summarise(sys.argv[1])
        print(f"{'kernel':40s} {'launches':>9s} {'total ms':>11s} {'share':>7s}")
        for k, n, ms, sh in res:
            print(f"{k:40s} {n:9d} {ms:11.3f} {100 * sh:6.2f}%")
        print(f"{'all':40s} {sum(r[1] for r in res):9d} {all_ms:11.3f}")
