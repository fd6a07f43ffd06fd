"""GB300 analogue of the paper's Table 1 and of its latency model (Sec. 1.6,
5.3, Eq. 3).

Measures the read-only bandwidth b of a thread-local-sum stream as a
function of occupancy (resident threads per SM) and of load parallelism
(ILP: independent 16-byte loads in flight per thread), and, with Little's
law as in Eq. 3, the memory latency each point implies:
    T = f * (bytes in flight) / b,
with bytes in flight = resident threads * ILP * 16 B (the paper's form with
8-byte loads is T = f N 8 B / b).  Prints a Markdown table.

Usage: python -m paper_1905_03136_gb300.microbench [--gib 4]
"""

import argparse
import os
import sys


def table(gib=4, clock_ghz=None):
    import torch
    import paper_1905_03136_gb300 as tsm
    from paper_1905_03136_gb300 import probe
    tsm.load()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    if clock_ghz is None:
        clock_ghz = 2.07
    buf = torch.empty(gib << 27, dtype=torch.float64, device="cuda")
    buf.fill_(1.0)
    rows = [("1 block, 4 warps", 1, 128)]
    for pct, threads_per_sm in ((6.25, 128), (12.5, 256), (25, 512), (50, 1024), (100, 2048)):
        if threads_per_sm <= 256:
            rows.append(("%g %%" % pct, sms, threads_per_sm))
        else:
            rows.append(("%g %%" % pct, sms * threads_per_sm // 256, 256))
    out = []
    for label, blocks, threads in rows:
        # every configuration here fits on the SMs at once (at most 2048
        # threads per SM), so all its loads can be in flight together
        vals = []
        for ilp in (1, 4, 16):
            b = probe.bandwidth(buf, mode=0, ilp=ilp, blocks=blocks, threads=threads)
            inflight = blocks * threads * ilp * 16.0
            vals.append((b, clock_ghz * 1e9 * inflight / (b * 1e9)))
        out.append((label, blocks, threads, vals))
    del buf
    return out, sms, clock_ghz


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gib", type=int, default=4)
    args = ap.parse_args()
    rows, sms, f = table(args.gib)
    print("| occupancy | CTAs x threads | ILP 1 GB/s | ILP 4 GB/s | ILP 16 GB/s | implied latency (cycles) ILP 1 / 4 / 16 |")
    print("|---|---|---|---|---|---|")
    bmax = max(v[0] for _, _, _, vals in rows for v in vals)

    def cell(v):
        # Little's law gives a latency only while the loads in flight do
        # not already saturate the memory system.
        if v[1] != v[1]:
            return "-"
        return "%.0f" % v[1] if v[0] < 0.8 * bmax else "sat."

    for label, blocks, threads, vals in rows:
        lat = " / ".join(cell(v) for v in vals)
        print("| %s | %d x %d | %.0f | %.0f | %.0f | %s |" % (label, blocks, threads, vals[0][0], vals[1][0],
                                                           vals[2][0], lat))
    print("\n(%d SMs; latency with f = %.2f GHz; \"sat.\": within 20 %% of the highest bandwidth, no latency implied)" % (sms, f))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
