"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import tebd  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    # Ground energy of the open critical transverse-field Ising chain (Sec. III.B:
    # exactly solvable at h = 1), from the closed form and the free-fermion form.
    rows = {}
    for L in (2, 8, 16, 32, 64):
        rows[str(L)] = {"closed_form": tebd.critical_ground_energy(L),
                        "free_fermion": tebd.free_fermion_ground_energy(L, 1.0)}
    with open(os.path.join(HERE, "tfim_critical_e0.json"), "w") as f:
        json.dump({"source": "Sec. III.B, spin-1/2 chain at h = h_c = 1; open boundaries",
                   "energies": rows}, f, indent=1)


if __name__ == "__main__":
    main()
