"""The networks the data-defined GPU executor runs are data in
paper_2007_03638_gb300/csrc/tnet.cu (ternary_netdef, binary_netdef: leaf legs,
roles and a pairwise contraction tree).  This CPU test reads that data,
contracts each tree pairwise with the executor's rule (a node keeps the legs
of one child that the other lacks) and compares the root with the oracle's
ascending map, so an edit to the network data fails here before any GPU run."""
import os
import re

import numpy as np
import pytest

from oracle import ternary as ot
from paper_2007_03638_gb300 import inputs as inp

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2007_03638_gb300", "csrc", "tnet.cu")
ROLE = {"ROLE_OP": "op", "ROLE_U": "u", "ROLE_UB": "ub", "ROLE_W": "w", "ROLE_WB": "wb"}


def _body(fn):
    src = open(SRC).read()
    i = src.index(f"NetDef {fn}(char side) {{")
    return src[i:src.index("\n}\n", i)]


def _netdefs():
    out = {}
    for side, body in re.findall(r"side == '([LCR])'\) \{(.*?)\n  \}", _body("ternary_netdef"), flags=re.S):
        legs_part, rest = body.split("d.role")
        legs = re.findall(r'"([^"]+)"', legs_part)
        roles = [ROLE[r] for r in re.findall(r"ROLE_[A-Z]+", rest.split("d.kids")[0])]
        kids = [(int(a), int(b)) for a, b in re.findall(r"\{(\d+), (\d+)\}", rest.split("d.kids")[1])]
        out[side] = (legs, roles, kids)
    return out


def test_three_networks_are_defined():
    assert sorted(_netdefs()) == ["C", "L", "R"]


@pytest.mark.parametrize("side", ["L", "C", "R"])
def test_network_data_matches_the_oracle(side):
    legs, roles, kids = _netdefs()[side]
    rng = np.random.default_rng(0)
    us, ws = inp.random_ternary_mera(2, 4, 1, seed=3, dtype=np.complex128)
    u, w = us[0], ws[0]
    c, cp = 2, 4
    op = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    u4, w4 = u.reshape(c, c, c, c), w.reshape(c, c, c, cp)
    arrays = {"op": op.reshape(c, c, c, c), "u": u4, "ub": u4.conj(), "w": w4, "wb": w4.conj()}
    assert roles[0] == "op" and len(legs) == len(roles) == 7
    # the leaves (legs and roles) are the oracle's network
    for i, (_, l, role) in enumerate(ot._network(side, u, w), start=1):
        assert (legs[i], roles[i]) == (l, role), (side, i)
    names = {}

    def sub(ls):
        return "".join(names.setdefault(x, chr(ord("a") + len(names))) for x in ls)

    val = {i: arrays[roles[i]] for i in range(len(legs))}
    lg = {i: legs[i].split() for i in range(len(legs))}
    for k, (a, b) in enumerate(kids):
        assert a < len(legs) + k and b < len(legs) + k  # children precede their node
        node = len(legs) + k
        free = [x for x in lg[a] if x not in lg[b]] + [x for x in lg[b] if x not in lg[a]]
        val[node] = np.einsum(f"{sub(lg[a])},{sub(lg[b])}->{sub(free)}", val[a], val[b])
        lg[node] = free
    root = len(legs) + len(kids) - 1
    out = ot.OUT_LEGS.split()
    assert sorted(lg[root]) == sorted(out)
    got = np.einsum(f"{sub(lg[root])}->{sub(out)}", val[root]).reshape(cp * cp, cp * cp)
    assert np.abs(got - ot.ascend_side(op, u, w, side)).max() < 1e-13


def _binary_netdefs():
    body = _body("binary_netdef")
    common = body[body.index("d.role"):]
    roles = [ROLE[r] for r in re.findall(r"ROLE_[A-Z]+", common.split("d.kids")[0])]
    kids = [(int(a), int(b)) for a, b in re.findall(r"\{(\d+), (\d+)\}", common.split("d.kids")[1])]
    out = {}
    for side, block in re.findall(r"side == '([LR])'\) \{(.*?)\n  \}", body, flags=re.S):
        legs = re.findall(r'"([^"]+)"', block.split("d.op_adj")[0])
        out[side] = (legs, roles, kids)
    return out


@pytest.mark.parametrize("side", ["L", "R"])
def test_binary_network_data_matches_the_oracle(side):
    from oracle import mera as om
    legs, roles, kids = _binary_netdefs()[side]
    assert roles[0] == "op" and len(legs) == len(roles) == 11 and len(kids) == 10
    rng = np.random.default_rng(1)
    us, ws = inp.random_mera(2, 4, 1, seed=5, dtype=np.complex128)
    u, w = us[0], ws[0]
    c, cp = 2, 4
    leaves, op_legs, out_legs, _ = om._network(side, u, w)
    # the leaves (legs and roles) are the oracle's network, in another order
    assert legs[0] == op_legs
    assert sorted(zip(legs[1:], roles[1:])) == sorted((l, r) for _, l, r in leaves)
    op = rng.standard_normal((c**3, c**3)) + 1j * rng.standard_normal((c**3, c**3))
    u4, w3 = u.reshape(c, c, c, c), w.reshape(c, c, cp)
    arrays = {"op": op.reshape((c,) * 6), "u": u4, "ub": u4.conj(), "w": w3, "wb": w3.conj()}
    names = {}

    def sub(ls):
        return "".join(names.setdefault(x, chr(ord("a") + len(names))) for x in ls)

    val = {i: arrays[roles[i]] for i in range(len(legs))}
    lg = {i: legs[i].split() for i in range(len(legs))}
    for k, (a, b) in enumerate(kids):
        assert a < len(legs) + k and b < len(legs) + k
        node = len(legs) + k
        free = [x for x in lg[a] if x not in lg[b]] + [x for x in lg[b] if x not in lg[a]]
        val[node] = np.einsum(f"{sub(lg[a])},{sub(lg[b])}->{sub(free)}", val[a], val[b])
        lg[node] = free
    root = len(legs) + len(kids) - 1
    out = out_legs.split()
    assert sorted(lg[root]) == sorted(out)
    got = np.einsum(f"{sub(lg[root])}->{sub(out)}", val[root]).reshape(cp**3, cp**3)
    assert np.abs(got - om.ascend_side(op, u, w, side)).max() < 1e-13
