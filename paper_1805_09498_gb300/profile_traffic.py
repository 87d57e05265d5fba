"""DRAM traffic per launch of the streaming kernels, from an ncu report.

    python -m paper_1805_09498_gb300.profile_traffic REPORT.ncu-rep \
        --frames-case 8000 --frames-full 20000 [--out profiles/ncu_traffic.json]

Reads `dram__bytes_read.sum + dram__bytes_write.sum` of the first captured
launch of k_estep and k_wcov (``ncu -i REPORT --page raw --csv``), scales
them from the profiled case to a full launch by the ratio of frames streamed
(traffic is proportional to the frames of a launch), and writes them with
the hash of the kernel sources, so that a reader (bench.py) can tell whether
the figures still describe the current kernels.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)


def sources_hash() -> str:
    """Hash of the CUDA sources and the C header (names and contents)."""
    h = hashlib.sha256()
    for d in (os.path.join(PKG, "csrc"), os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


def read_report(path: str):
    out = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr = rows[0]
    name = hdr.index("Kernel Name")
    rd, wr = hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")
    unit_rd, unit_wr = rows[1][rd], rows[1][wr]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    res = []
    for r in rows[2:]:
        b = float(r[rd].replace(",", "")) * scale[unit_rd] + float(r[wr].replace(",", "")) * scale[unit_wr]
        res.append((r[name], b))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("report")
    ap.add_argument("--frames-case", type=float, required=True)
    ap.add_argument("--frames-full", type=float, required=True)
    ap.add_argument("--how", default="")
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "ncu_traffic.json"))
    a = ap.parse_args()
    ratio = a.frames_full / a.frames_case
    kernels = {}
    for name, b in read_report(a.report):
        for k in ("k_estep", "k_wcov"):
            if name.startswith(f"void {k}<") and k not in kernels:
                kernels[k] = {"kernel": name, "dram_bytes_small_case": b, "dram_bytes_per_launch": b * ratio}
    doc = {"csrc_sha": sources_hash(), "how": a.how, "frames_ratio": ratio, "kernels": kernels}
    with open(a.out, "w") as fh:
        json.dump(doc, fh, indent=1)
    print(json.dumps(doc, indent=1))


if __name__ == "__main__":
    main()
