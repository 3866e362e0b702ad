"""Write the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

rademacher_signs.txt: start-vector entries (seed, b, l, i, value) for seeds 0
and 12345 -- the splitmix64-counter Rademacher generator that both the oracle
and the CUDA path implement from the published splitmix64 definition.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import kpm  # noqa: E402


def main():
    rows = []
    for seed in (0, 12345):
        for b in (0, 3):
            for l in (0, 1, 5, 63, 64, 200):
                for i in range(16):
                    rows.append((seed, b, l, i, int(kpm.rademacher(seed, b, l, i))))
    with open(os.path.join(HERE, "rademacher_signs.txt"), "w") as f:
        f.write("# seed b l i value  -- written by tests/golden/make_golden.py from oracle.kpm\n")
        for r in rows:
            f.write(" ".join(str(x) for x in r) + "\n")


if __name__ == "__main__":
    main()
