"""Write touring_digests.txt: digests of the oracle's longest-first touring
TP sets of the 4096-graph batch (seeded structured CFGs) and of the
120-vertex CFG, for the full-size GPU parity test.

Calls only the oracle (oracle/).  Single-threaded it takes about 20 minutes,
so the GPU test compares against these stored digests instead of running it.

    python tests/golden/make_touring_digests.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2210_16998_gb300 import cfggen as G  # noqa: E402
from tests.helpers import touring_digest_update as digest_update  # noqa: E402

GROUP = 64


def main():
    lines = ["# digests of the oracle's longest-first touring TP sets",
             "# written by tests/golden/make_touring_digests.py (oracle only)",
             "# name first_graph graphs test_paths tp_vertices sha256_16"]
    cfgs = G.batch_cfgs(4096, G.BATCH_SEED0)
    for g0 in range(0, len(cfgs), GROUP):
        h = hashlib.sha256()
        T = V = 0
        for c in cfgs[g0:g0 + GROUP]:
            r = oracle.run_cfg(c, test_paths=False, greedy=True)
            digest_update(h, r.gtp_offsets, r.gtp_vertices)
            T += len(r.gtp_offsets) - 1
            V += int(r.gtp_offsets[-1])
        lines.append(f"batch4096 {g0} {min(GROUP, len(cfgs) - g0)} {T} {V} {h.hexdigest()[:16]}")
        print(lines[-1], flush=True)
    r = oracle.run_cfg(G.config3_cfg(), test_paths=False, greedy=True)
    h = hashlib.sha256()
    digest_update(h, r.gtp_offsets, r.gtp_vertices)
    lines.append(f"config3 0 1 {len(r.gtp_offsets) - 1} {int(r.gtp_offsets[-1])} {h.hexdigest()[:16]}")
    with open(os.path.join(HERE, "touring_digests.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
