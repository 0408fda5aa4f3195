"""Write the stored expected values of tests/golden/ from the FP64 oracle.

Only oracle/ is called.  roundtrip_defect.json holds, per truncation of the
octahedral grid, the quadrature defect E = max_m max_{n,n'} |sum over the
rings that drop m of w_k P_n^m P_n'^m| (oracle.roundtrip_defect): the most
by which direct(inverse(a)) can differ from a per unit of sum|a|.  Computing
it at TCo1279 takes minutes, so the full-size round-trip test reads it here.

    python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    out = {}
    for T in (79, 639, 1279):
        e, _ = oracle.roundtrip_defect(T, 0, T + 1)
        out[str(T)] = e
        print(T, e, flush=True)
    with open(os.path.join(HERE, "roundtrip_defect.json"), "w") as f:
        json.dump({"grid": "octahedral O(T+1)", "source": "oracle.roundtrip_defect", "defect": out}, f, indent=1)


if __name__ == "__main__":
    main()
