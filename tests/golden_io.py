"""Readers for the text fixtures under tests/golden/ (closed-form values)."""
import math
import os
from fractions import Fraction

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _eval(expr: str) -> float:
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def lobatto_rules():
    """{M: (nodes, weights)} from lobatto_rules.txt."""
    out = {}
    for line in _lines("lobatto_rules.txt"):
        m, nodes, weights = [p.strip() for p in line.split("|")]
        out[int(m)] = ([_eval(e) for e in nodes.split(",")], [_eval(e) for e in weights.split(",")])
    return out


def lobatto_iiia_m3():
    return [[float(Fraction(t)) for t in line.split()] for line in _lines("lobatto_iiia_M3.txt")]


def pade_numerators():
    out = {}
    for line in _lines("pade_lobatto_iiia.txt"):
        m, coeffs = [p.strip() for p in line.split("|")]
        out[int(m)] = [float(Fraction(c.strip())) for c in coeffs.split(",")]
    return out


def _family_lines(name):
    for line in _lines(name):
        head, rest = line.split("|", 1)
        fam, m = head.split()
        yield fam, int(m), rest


def radau_legendre_rules():
    """{(family, M): (nodes, weights)} from radau_legendre_rules.txt."""
    out = {}
    for fam, m, rest in _family_lines("radau_legendre_rules.txt"):
        nodes, weights = [p.strip() for p in rest.split("|")]
        out[(fam, m)] = ([_eval(e) for e in nodes.split(",")], [_eval(e) for e in weights.split(",")])
    return out


def collocation_tableaus():
    """{(family, M): A} from collocation_tableaus.txt."""
    out = {}
    for fam, m, rest in _family_lines("collocation_tableaus.txt"):
        out[(fam, m)] = [[_eval(e) for e in row.split(",")] for row in rest.split(";")]
    return out


def pade_radau_gauss():
    """{(family, M): (numerator, denominator)} coefficient lists, ascending powers."""
    out = {}
    for fam, m, rest in _family_lines("pade_radau_gauss.txt"):
        num, den = [p.strip() for p in rest.split("|")]
        out[(fam, m)] = ([float(Fraction(c.strip())) for c in num.split(",")],
                         [float(Fraction(c.strip())) for c in den.split(",")])
    return out
