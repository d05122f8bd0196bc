"""Writes opcount_slab128.json: the algorithmic FP64 work of one thermochemistry step
per cell of the 128^3 slab workload, counted by the CPU oracle's operation counter.

The counts are the method's own operations (every add, multiply, divide, sqrt, exp,
log and pow of the substeps and iterations the scheme performs, Sec. 6.1), averaged
over a seeded random sample of the slab's cells, for the paper's sequential scheme
(mode 0) and the coupled implicit scheme (mode 1).  The benchmark multiplies them by
the cells one launch processes to state the roofline numerator.

Run from the repository root:  python tests/golden/make_opcount.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthgen  # noqa: E402

SAMPLE = 8192


def main():
    c = synthgen.slab()
    idx = np.sort(np.random.default_rng(12345).choice(c["n"].size, SAMPLE, replace=False))
    sub = synthgen.subset(c, idx)
    out = {"_comment": "Per-cell algorithmic FP64 operation counts of one step (dt = 1e4 yr) on the 128^3 slab, "
                       "averaged over %d seeded random cells; written by tests/golden/make_opcount.py from the "
                       "oracle's operation counter." % SAMPLE,
           "workload": "slab128", "dt_s": synthgen.DT_1E4YR, "sample": SAMPLE}
    for mode in (0, 1):
        oc = oracle.opcount(sub, synthgen.DT_1E4YR, oracle.default_params(mode=mode))
        res = oc.pop("result")
        out["mode%d" % mode] = {k: v / SAMPLE for k, v in oc.items()}
        out["mode%d" % mode]["nsub_mean"] = float(np.mean(res["nsub"]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "opcount_slab128.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
