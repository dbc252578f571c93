"""DRAM traffic record of the 2-D step kernels: profiles/traffic.json.

bench.py reports the dominant kernel's DRAM bytes per launch from this record,
but only while the record was captured on the step-kernel sources in the tree
(their hash is stored with it). This tool writes the record from ncu CSVs
of the benchmark workload, e.g. (on one GB300, from the repository root,
B = "python bench.py --nt 16 --steps 1 --warmup 3 --no-cpu-baseline
--no-e2e --profile-region"):

    $B --variant V > plain.log && \
    ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \
        --clock-control none -k regex:K -s 2 -c 2 --profile-from-start off \
        --csv --log-file traffic_V_K.csv $B --variant V

for (V, K) = (full, k_fwd_step): the forward step of the offset-Hessian run
(fused, or with a split variant the plain step); (full, k_offh_level): its
offset-Hessian sums (split variants); (full, k_bwd_step): the backward step;
(plain, k_fwd_step): the plain forward step. Then

    python -m paper_1406_1864_gb300.traffic traffic_*.csv

Each kernel's bytes per launch are the mean over its captured launches. The
plain step captured in the offset-Hessian run is recorded as
"k_fwd_step (full)".
"""
from __future__ import annotations

import csv
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "profiles", "traffic.json")
WORKLOAD = "dipping_300x1000_96shots"
CAPTURES = {
    "k_fwd_step<offset Hessian>": "profiles/k_fwd_step_offset_hessian_dipping_300x1000_96shots.md",
    "k_fwd_step (full)": "profiles/k_fwd_step_dipping_300x1000_96shots.md",
    "k_offh_level": "profiles/k_offh_level_dipping_300x1000_96shots.md",
    "k_fwd_step": "profiles/k_fwd_step_dipping_300x1000_96shots.md",
    "k_bwd_step": "profiles/k_bwd_step_dipping_300x1000_96shots.md",
}


def key_of(kernel_name: str) -> str | None:
    """Record key of a demangled step-kernel name: the forward step's third
    template argument is 1 with the offset Hessian fused."""
    if kernel_name.startswith("void k_bwd_step<"):
        return "k_bwd_step"
    if kernel_name.startswith("void k_offh_level<"):
        return "k_offh_level"
    if kernel_name.startswith("void k_fwd_step<"):
        args = kernel_name[len("void k_fwd_step<"):].split(",")
        return "k_fwd_step<offset Hessian>" if args[2].strip() == "1" else "k_fwd_step"
    return None


def read_csv(path: str) -> dict:
    """{key: (kernel name, [bytes of each launch])} from an ncu --csv log."""
    per = {}
    with open(path) as f:
        rows = [ln for ln in f if ln.startswith('"')]
    launches = {}
    for r in csv.DictReader(rows):
        k = key_of(r["Kernel Name"])
        if k is None:
            continue
        d = launches.setdefault((k, r["ID"]), {"name": r["Kernel Name"]})
        d[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    for (k, _), d in launches.items():
        b = d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0)
        per.setdefault(k, (d["name"], []))[1].append(b)
    return per


def main(paths):
    sys.path.insert(0, ROOT)
    import bench
    rec = {}
    for p in paths:
        full = "_full_" in os.path.basename(p)
        for k, (name, bs) in read_csv(p).items():
            key = "k_fwd_step (full)" if (k == "k_fwd_step" and full) else k
            rec[key] = {"kernel": name, "workload": WORKLOAD, "source_hash": bench.kernel_source_hash(),
                        "bytes_per_launch": sum(bs) / len(bs), "launches": len(bs), "capture": CAPTURES.get(key)}
    if "k_bwd_step" not in rec:
        raise SystemExit(f"no launches of k_bwd_step in {paths}")
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main(sys.argv[1:])
