"""Short markdown summaries of ncu's CSV output (`ncu --csv --log-file FILE ...`),
the form in which kernel measurements are kept next to the code.

  launches  per kernel: launches, total and mean device time, share of the total
            (from a `--metrics gpu__time_duration.sum` launch list; cold-cache and
            serialised, so the shares are what compare with a timed run);
  metrics   per kernel: the mean per launch of every captured metric and, where the
            DRAM byte counters were captured, the traffic per launch and (with the
            duration) its rate against the measured HBM copy bandwidth;
  phases    one tuned step of the library from a launch list: the per-launch mean of
            each of its kernels, grouped by the phase of the hot path they belong to,
            and each phase's share of the step's serialised kernel time.

Usage:
    python -m paper_2406_06488_gb300.ncu_summary launches FILE.csv
    python -m paper_2406_06488_gb300.ncu_summary metrics FILE.csv [--peaks MEASURED_PEAKS.json]
    python -m paper_2406_06488_gb300.ncu_summary phases FILE.csv

Reads only the CSV (and the peaks file); it runs nothing on a GPU.
"""
import argparse
import csv
import io
import json
from collections import OrderedDict

DURATION = "gpu__time_duration.sum"
DRAM_READ = "dram__bytes_read.sum"
DRAM_WRITE = "dram__bytes_write.sum"

_TIME_NS = {"ns": 1.0, "nsecond": 1.0, "us": 1e3, "usecond": 1e3, "ms": 1e6, "msecond": 1e6, "s": 1e9, "second": 1e9}
_BYTES = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}


def read_rows(text):
    """The CSV records of ncu's output (its ==PROF== / ==WARNING== lines skipped)."""
    lines = [ln for ln in text.splitlines() if ln.strip() and not ln.startswith("==")]
    return list(csv.DictReader(io.StringIO("\n".join(lines))))


def kernel_name(full):
    """A kernel's name without its return type and parameter list (template arguments
    kept; a stray '>' such as that of a truncated '<unnamed>' is tolerated)."""
    name = full[5:] if full.startswith("void ") else full
    depth = 0
    for i, ch in enumerate(name):
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth = max(depth - 1, 0)
        elif ch == "(" and depth == 0 and i > 0:
            return name[:i]
    return name


def _value(row):
    return float(row["Metric Value"].replace(",", ""))


def _launches(rows):
    """OrderedDict launch id -> (kernel, {metric: (value, unit)}), in capture order."""
    out = OrderedDict()
    for r in rows:
        lid = (r.get("Process ID", ""), r["ID"])
        entry = out.setdefault(lid, (kernel_name(r["Kernel Name"]), {}))
        entry[1][r["Metric Name"]] = (_value(r), r.get("Metric Unit", ""))
    return out


def _ns(v):
    value, unit = v
    return value * _TIME_NS.get(unit, 1.0)


def _bytes(v):
    value, unit = v
    return value * _BYTES.get(unit, 1.0)


def launch_table(rows):
    """[(kernel, launches, total_us, mean_us, share)] sorted by total time, largest first."""
    per = OrderedDict()
    for kern, m in _launches(rows).values():
        if DURATION not in m:
            continue
        n, tot = per.get(kern, (0, 0.0))
        per[kern] = (n + 1, tot + _ns(m[DURATION]) / 1e3)
    grand = sum(t for _, t in per.values()) or 1.0
    table = [(k, n, t, t / n, t / grand) for k, (n, t) in per.items()]
    table.sort(key=lambda x: -x[2])
    return table


def metric_table(rows, hbm_gbs=None):
    """{kernel: {"launches": n, metric: mean value, ..., "traffic_bytes": ..., "dram_gbs": ...,
    "dram_frac": ...}} with the means taken per launch."""
    acc = OrderedDict()
    for kern, m in _launches(rows).values():
        a = acc.setdefault(kern, {"launches": 0, "_sums": OrderedDict(), "_traffic": [], "_ns": []})
        a["launches"] += 1
        for name, v in m.items():
            a["_sums"][name] = a["_sums"].get(name, 0.0) + v[0]
        if DRAM_READ in m and DRAM_WRITE in m:
            a["_traffic"].append(_bytes(m[DRAM_READ]) + _bytes(m[DRAM_WRITE]))
            if DURATION in m:
                a["_ns"].append(_ns(m[DURATION]))
    out = OrderedDict()
    for kern, a in acc.items():
        d = OrderedDict(launches=a["launches"])
        for name, s in a["_sums"].items():
            d[name] = s / a["launches"]
        if a["_traffic"]:
            d["traffic_bytes"] = sum(a["_traffic"]) / len(a["_traffic"])
            if a["_ns"] and len(a["_ns"]) == len(a["_traffic"]):
                gbs = sum(a["_traffic"]) / sum(a["_ns"])   # bytes per ns = GB/s
                d["dram_gbs"] = gbs
                if hbm_gbs:
                    d["dram_frac"] = gbs / hbm_gbs
        out[kern] = d
    return out


def launches_markdown(table):
    lines = ["| kernel | launches | total us | mean us | share |", "|---|---:|---:|---:|---:|"]
    for k, n, t, mean, share in table:
        lines.append("| %s | %d | %.1f | %.1f | %.1f%% |" % (k, n, t, mean, 100.0 * share))
    return "\n".join(lines)


def metrics_markdown(table):
    lines = []
    for kern, d in table.items():
        lines.append("%s (%d launch%s)" % (kern, d["launches"], "" if d["launches"] == 1 else "es"))
        lines.append("")
        lines.append("| counter | mean per launch |")
        lines.append("|---|---:|")
        for name, v in d.items():
            if name == "launches":
                continue
            lines.append("| %s | %.6g |" % (name, v))
        lines.append("")
    return "\n".join(lines).rstrip()


# the tuned path's kernels by phase (the plain path's k_contract_simt, k_build_simt,
# k_norms and k_pack<0>, and the bench's own kernels, are not part of a tuned step)
PHASES = [
    ("contraction", ["k_contract_tc", "k_contract_tc2", "k_contract_tm"]),
    ("relabeling draws (side stream)", ["k_masks", "k_masks_lanes"]),
    ("block build", ["k_split_rows", "k_build_tc"]),
    ("centring / packing", ["k_blocksums", "k_rowsum_reduce", "k_center_u", "k_center_r", "k_pack<1>"]),
    ("combination", ["k_combine_stats", "k_combine_count", "k_batch_status", "k_reset_counts"]),
    ("recomputation of flagged statistics", ["k_refine_packed", "k_refine_packed_finish", "k_refine_w",
                                             "k_refine_rows", "k_refine_finish"]),
]


def _short(kernel):
    """A kernel name without its namespaces ('ept::<unnamed>::k_pack<1>' -> 'k_pack<1>')."""
    name = kernel.replace("<unnamed>::", "").replace("unnamed>::", "")
    cut = name.split("<")[0].rfind("::")
    return name[cut + 2:] if cut >= 0 else name


def phase_table(rows):
    """[(phase, kernels, us, share)]: per phase the sum of its kernels' per-launch means."""
    means = {_short(k): mean for k, n, t, mean, share in launch_table(rows)}
    out = []
    for phase, kernels in PHASES:
        present = [k for k in kernels if k in means]
        if present:
            out.append((phase, present, sum(means[k] for k in present)))
    total = sum(us for _, _, us in out) or 1.0
    return [(ph, ks, us, us / total) for ph, ks, us in out]


def phases_markdown(table):
    lines = ["| phase | kernels | us | share of the serialised step |", "|---|---|---:|---:|"]
    for ph, ks, us, share in table:
        lines.append("| %s | %s | %.1f | %.1f %% |" % (ph, ", ".join(ks), us, 100.0 * share))
    lines.append("| total | | %.1f | |" % sum(us for _, _, us, _ in table))
    return "\n".join(lines)


def summarise(mode, text, hbm_gbs=None):
    """The markdown summary of ncu CSV text: mode 'launches', 'metrics' or 'phases'."""
    rows = read_rows(text)
    if mode == "launches":
        return launches_markdown(launch_table(rows))
    if mode == "metrics":
        return metrics_markdown(metric_table(rows, hbm_gbs))
    if mode == "phases":
        return phases_markdown(phase_table(rows))
    raise ValueError("mode must be 'launches', 'metrics' or 'phases'")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("mode", choices=["launches", "metrics", "phases"])
    ap.add_argument("csv")
    ap.add_argument("--peaks", default=None, help="MEASURED_PEAKS.json (hbm_gbs) for the DRAM fraction")
    args = ap.parse_args(argv)
    hbm = None
    if args.peaks:
        with open(args.peaks) as f:
            hbm = json.load(f).get("hbm_gbs")
    with open(args.csv) as f:
        print(summarise(args.mode, f.read(), hbm))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
