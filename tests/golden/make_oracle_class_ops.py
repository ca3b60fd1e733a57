#!/usr/bin/env python3
"""Write oracle_class_ops.json: the oracle's operation counts per angular-momentum class.

For every class (la lb | lc ld), l <= 4, the OS/HGP oracle's instrumented counter
(oracle.class_ops) gives the operations of one primitive quartet (set-up, Boys, VRR,
contraction) and of one contracted quartet (HRR, digestion of one density into J and K).
The benchmark multiplies them by the primitive and contracted quartets each class launch
evaluates to report its roofline fraction in oracle operations.  Calls only oracle/.

    python tests/golden/make_oracle_class_ops.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_class_ops.json")


def table():
    rows = {}
    for la in range(5):
        for lb in range(5):
            for lc in range(5):
                for ld in range(5):
                    pp, pq = oracle.class_ops(la, lb, lc, ld, nD=1)
                    rows[f"{la}{lb}{lc}{ld}"] = {"per_prim": sum(pp.values()), "hrr": pq["hrr"],
                                                 "digest_per_density": pq["digest"]}
    return {"what": "operations of the OS/HGP oracle per class (la lb|lc ld): per primitive quartet "
                    "(set-up, Boys, VRR, contraction), per contracted quartet the transfer relations and "
                    "the digestion of one density into J and K (8 ordered quartets x 4 per value)",
            "counted_by": "oracle.class_ops (tests/test_oracle_ops.py pins the counter)",
            "classes": rows}


if __name__ == "__main__":
    t = table()
    with open(OUT, "w") as f:
        f.write("{\"what\": %s,\n \"counted_by\": %s,\n \"classes\": {\n" % (json.dumps(t["what"]),
                                                                         json.dumps(t["counted_by"])))
        f.write(",\n".join("  \"%s\": %s" % (k, json.dumps(v, sort_keys=True)) for k, v in sorted(t["classes"].items())))
        f.write("\n}}\n")
    print(OUT)
