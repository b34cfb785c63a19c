#!/usr/bin/env python
"""DRAM traffic of the pair-tile kernel on the bench workload, for the
``traffic`` field of bench.py's roofline.

Runs the bench's default workload once without a profiler (it must exit 0),
then once under ncu collecting only dram__bytes_read.sum,
dram__bytes_write.sum and gpu__time_duration.sum (one pass per launch) for
the k_pair_tile launches, and writes ncu_traffic.json: the bytes per launch
(the mean over the captured launches), the workload and the SHA-256 of the
kernel's sources.  bench.py uses the figure only while both still match.
Run on a GPU machine:  python ncu_traffic.py
"""
import csv
import hashlib
import io
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["kernels_pairs.cu", "engine.cuh", "philox.cuh", "fp.cuh"]
BENCH = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "1", "--profile-steps", "1",
         "--e2e-steps", "0", "--no-cpu-baseline", "--extras", "0", "--autotune", "0"]
OUT = os.path.join(ROOT, "ncu_traffic.json")


def source_hash():
    h = hashlib.sha256()
    for f in SOURCES:
        with open(os.path.join(ROOT, "paper_1208_0961_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def main():
    plain = subprocess.run(BENCH, capture_output=True, text=True)
    if plain.returncode != 0:
        sys.stderr.write(plain.stdout + plain.stderr)
        return plain.returncode
    workload = json.loads(plain.stdout.strip().splitlines()[-1])["config"]["workload"]
    log = os.path.join(ROOT, "gpurun_out", "ncu_traffic.csv")
    os.makedirs(os.path.dirname(log), exist_ok=True)
    cmd = ["ncu", "--metrics", "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum",
           "--clock-control", "none", "-k", "regex:k_pair_tile", "--csv", "--log-file", log] + BENCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout[-4000:] + r.stderr[-4000:])
        return r.returncode
    with open(log) as f:
        lines = f.read().splitlines()
    head = next(k for k, ln in enumerate(lines) if ln.startswith('"ID"'))
    rows = list(csv.DictReader(io.StringIO("\n".join(lines[head:]))))
    per = {}
    for row in rows:
        if "k_pair_tile" not in row.get("Kernel Name", ""):
            continue
        key = row["ID"]
        val = float(row["Metric Value"].replace(",", ""))
        unit = row.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-9, "usecond": 1e-6,
                 "msecond": 1e-3}.get(unit, 1)
        per.setdefault(key, {})[row["Metric Name"]] = val * scale
    launches = [v for v in per.values() if "dram__bytes_read.sum" in v]
    if not launches:
        sys.stderr.write("no k_pair_tile launch captured\n")
        return 1
    nbytes = sum(v["dram__bytes_read.sum"] + v.get("dram__bytes_write.sum", 0.0) for v in launches) / len(launches)
    rec = {"k_pair_tile": {"dram_bytes_per_launch": nbytes, "launches": len(launches), "workload": workload,
                           "source_sha256": source_hash(),
                           "metrics": "dram__bytes_read.sum + dram__bytes_write.sum, one pass per launch",
                           "command": " ".join(["ncu"] + cmd[1:9] + ["gpurun_out/ncu_traffic.csv", "python",
                                                                     "bench.py"] + BENCH[2:])}}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))
    return 0


if __name__ == "__main__":
    sys.exit(main())
