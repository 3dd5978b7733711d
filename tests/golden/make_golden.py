"""Write tests/golden/polyene8.txt from the CPU oracle only.

Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import hci_inputs as hi  # noqa: E402
import oracle  # noqa: E402


def main():
    inst = hi.ppp_polyene(8)
    fci = oracle.hci(inst, 0.0)
    r4 = oracle.hci(inst, 1e-4)
    with open(os.path.join(HERE, "polyene8.txt"), "w") as fh:
        fh.write("# 8-site PPP polyene (8e,8o), Hueckel MO basis, values from the CPU oracle\n")
        fh.write("# (written by tests/golden/make_golden.py; FCI = HCI at eps1 = 0)\n")
        fh.write(f"E_fci = {fci['E']:.15f}\n")
        fh.write(f"nV_fci = {len(fci['keys'])}\n")
        fh.write(f"E_eps1e-4 = {r4['E']:.15f}\n")
        fh.write(f"nV_eps1e-4 = {len(r4['keys'])}\n")
        fh.write(f"iters_eps1e-4 = {len(r4['history'])}\n")


if __name__ == "__main__":
    main()
