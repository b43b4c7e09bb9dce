"""Generate csrc/dvm_sets.h: compile-time velocity sets for the kernels.

For each listed DVM of the paper (2D tables as printed, or the (x, z)
marginal of a 3D table) the header lists the pair representatives +e of the
+-e pairs (e_y > 0, or e_y = 0 and e_x > 0) and whether a rest velocity is
present.  Weights are not in the header: they stay run-time arguments of
lbm_create, so any weight vector on one of these velocity sets uses the
specialised kernel.

    python -m paper_1510_08886_gb300.gen_dvm_sets          # rewrite the header
    python -m paper_1510_08886_gb300.gen_dvm_sets --check  # exit 1 if stale
"""
import itertools
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "dvm_sets.h")

# (C++ identifier, table name, marginal?)
SETS = [("D2V16", "D2V16", False), ("D2V32", "D2V32", False), ("D2V33", "D2V33", False),
        ("D2V53", "D3V107", True), ("D2V40", "D3V96", True), ("D2V48", "D3V112", True)]


def _orbit(rep):
    D = len(rep)
    out = set()
    for perm in itertools.permutations(rep):
        for signs in itertools.product((1, -1), repeat=D):
            out.add(tuple(s * p for s, p in zip(signs, perm)))
    return out


def velocity_set(table, marginal):
    vels = set()
    for rep, _, _ in table["groups"]:
        vels |= _orbit(rep)
    if marginal:
        vels = {(v[0], v[2]) for v in vels}
    return vels


def pairs_of(vels):
    rest = (0, 0) in vels
    pos = sorted((v for v in vels if v[1] > 0 or (v[1] == 0 and v[0] > 0)),
                 key=lambda v: (v[0] * v[0] + v[1] * v[1], -v[1], -v[0]))
    assert len(pos) * 2 + rest == len(vels)
    return rest, pos


def render():
    sys.path.insert(0, os.path.dirname(HERE))
    from lbm_inputs import DVM_TABLES
    out = ["// Generated by paper_1510_08886_gb300/gen_dvm_sets.py from the paper's DVM",
           "// tables (App. A, App. B): compile-time +-e pair representatives of the",
           "// velocity sets with register-resident specialised kernels.  Do not edit.",
           "#pragma once", "", "namespace lbm {", ""]
    for ident, tname, marg in SETS:
        rest, pos = pairs_of(velocity_set(DVM_TABLES[tname], marg))
        src = f"(x, z) marginal of {DVM_TABLES[tname]['symbol']}" if marg else DVM_TABLES[tname]["symbol"]
        out.append(f"// {src}: V = {len(pos) * 2 + rest}")
        out.append(f"struct Set{ident} {{")
        out.append(f"    static constexpr int R = {int(rest)}, P = {len(pos)};")
        out.append("    static constexpr int ex[P] = {" + ", ".join(str(v[0]) for v in pos) + "};")
        out.append("    static constexpr int ey[P] = {" + ", ".join(str(v[1]) for v in pos) + "};")
        out.append("};")
        out.append("")
    out.append("}  // namespace lbm")
    out.append("")
    return "\n".join(out)


def main():
    txt = render()
    if "--check" in sys.argv:
        cur = open(HEADER).read() if os.path.exists(HEADER) else ""
        sys.exit(0 if cur == txt else 1)
    with open(HEADER, "w") as fh:
        fh.write(txt)
    print(HEADER)


if __name__ == "__main__":
    main()
