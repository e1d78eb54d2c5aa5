"""Algorithmic FP64 flop count of the per-pair integration, from the oracle.

Runs the oracle's own binned search on a workload, then its per-pair
integration with the flop-counting scalar (+ - * / sqrt count one each; the
slave element's auxiliary plane and LM coefficients are element-level
precomputation and not counted).  Prints one JSON line; the benchmark's
roofline numerator for the integration kernel is this count.

    python -m oracle.count_flops planar_2000x1733
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2202_03933_gb300 import inputs  # noqa: E402


def main(name: str) -> dict:
    itf = inputs.by_name(name)
    t0 = time.time()
    s, m = oracle.search_binned(itf)
    o = oracle.make_opts(lm=itf.lm, delta=itf.delta, n_threads=os.cpu_count() or 1)
    flops = oracle.count_pair_flops(itf, s, m, o)
    return {"workload": name, "pairs": int(s.size), "flops": int(flops),
            "flops_per_pair": flops / max(s.size, 1), "seconds": round(time.time() - t0, 1)}


if __name__ == "__main__":
    for n in sys.argv[1:] or ["planar_2000x1733"]:
        print(json.dumps(main(n)))
