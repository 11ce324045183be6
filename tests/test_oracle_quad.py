"""Pins of the oracle's quad-direction cells (Sec. 3.2, Algorithm 1) against
hand-placed sources whose cell sets were worked out from the layout of the
HEALPix base faces (``tests/golden/quad_cells.txt``, each case with its
derivation), and a mutation check: each plausible misreading of the rule,
planted in a copy of the oracle's C source and compiled on the CPU, must
disagree with at least one of those cases."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "quad_cells.txt")
GOLDEN_COS = os.path.join(HERE, "golden", "quad_cells_cos.txt")
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "hlc_oracle.c")


def _cases(path=GOLDEN):
    out = []
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        lhs, rhs = ln.split(":")
        ra, dec, r, L = lhs.split()
        out.append((float(ra), float(dec), float(r), int(L), [int(x) for x in rhs.split()]))
    return out


CASES = _cases()
CASES_COS = _cases(GOLDEN_COS)


def test_golden_file_covers_the_rule():
    assert len(CASES) >= 12
    counts = {len(c[4]) for c in CASES}
    assert {1, 2, 4, 5} <= counts          # one cell up to five distinct cells
    assert any(c[1] > 89 for c in CASES) and any(c[1] < -89 for c in CASES)  # clamps
    assert any(c[0] < 0.01 for c in CASES) and any(c[0] > 359.99 for c in CASES)  # wraps


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}_{c[1]}_{c[2]}_L{c[3]}" for c in CASES])
def test_quad_cells_equal_hand_placed_sets(case):
    ra, dec, r, L, want = case
    cells, cnt = O.quad_cells([ra], [dec], r, L)
    assert cells[0, :cnt[0]].tolist() == want
    assert np.all(cells[0, cnt[0]:] == np.iinfo(np.uint64).max)


@pytest.mark.parametrize("case", CASES_COS,
                         ids=[f"{c[0]}_{c[1]}_{c[2]}_L{c[3]}" for c in CASES_COS])
def test_cos_variant_cells_equal_hand_placed_sets(case):
    """The variant with R_A = R / cos(dec), beside the literal reading."""
    ra, dec, r, L, want = case
    cells, cnt = O.quad_cells([ra], [dec], r, L, cosdec=True)
    assert cells[0, :cnt[0]].tolist() == want


def test_the_two_readings_differ_where_cos_dec_matters():
    lit = {c[:4]: c[4] for c in CASES}
    cos = {c[:4]: c[4] for c in CASES_COS}
    common = set(lit) & set(cos)
    assert any(lit[k] != cos[k] for k in common)           # Dec 60 and the pole
    assert all(lit[k] == cos[k] for k in common if k[1] == 0.0)  # equator: equal


# Each misreading as a textual change of the oracle source: (old, new).  Every
# `old` must occur exactly once, so a reworded oracle fails loudly here.
MUTANTS = {
    "R_in_radians": [("double R = r_arcsec / 3600.0;",
                      "double R = r_arcsec * (M_PI / 648000.0);")],
    "R_halved": [("double R = r_arcsec / 3600.0;", "double R = r_arcsec / 7200.0;")],
    "R_doubled": [("double R = r_arcsec / 3600.0;", "double R = r_arcsec / 1800.0;")],
    "R_in_arcmin": [("double R = r_arcsec / 3600.0;", "double R = r_arcsec / 60.0;")],
    "dec_minus_typo": [("double dec_minus = dec - R;", "double dec_minus = dec + R;")],
    "wrap_by_c_fmod": [("  double y = x;\n  if (y < 0.0)",
                        "  double y = fmod(x, 360.0);\n  return y;\n  if (y < 0.0)")],
    "no_wrap": [("  double y = x;\n  if (y < 0.0)", "  double y = x;\n  return y;\n  if (y < 0.0)")],
    "no_clamp": [("if (dec_plus > 90.0) dec_plus = 90.0;", ""),
                 ("if (dec_minus < -90.0) dec_minus = -90.0;", "")],
    "reflect_through_pole": [
        ("p[4] = orc_ang2pix(ra, dec_plus, order);",
         "p[4] = dec + R > 90.0 ? orc_ang2pix(wrap_ra(ra + 180.0), 180.0 - (dec + R), order)"
         " : orc_ang2pix(ra, dec_plus, order);"),
        ("p[3] = orc_ang2pix(ra, dec_minus, order);",
         "p[3] = dec - R < -90.0 ? orc_ang2pix(wrap_ra(ra + 180.0), -180.0 - (dec - R), order)"
         " : orc_ang2pix(ra, dec_minus, order);")],
    "ra_shift_over_cos_dec": [
        ("double RA = cosdec ? ra_shift_cos(R, dec) : R;", "double RA = ra_shift_cos(R, dec);")],
    "no_dedup": [("if (m == 0 || p[i] != out[m - 1]) out[m++] = p[i];", "out[m++] = p[i];")],
}


def _build_mutant(tmp_path, name, edits):
    src = open(ORACLE_SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    cdir = tmp_path / name
    cdir.mkdir()
    (cdir / "hlc_oracle.c").write_text(src)
    hdr = os.path.join(os.path.dirname(ORACLE_SRC), "hlc_oracle.h")
    (cdir / "hlc_oracle.h").write_text(open(hdr).read())
    so = cdir / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(cdir / "hlc_oracle.c"), "-lm"])
    lib = C.CDLL(str(so))
    lib.orc_quad_cells.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int,
                                   C.POINTER(C.c_uint64)]
    lib.orc_quad_cells.restype = C.c_int
    lib.orc_quad_cells_cos.argtypes = lib.orc_quad_cells.argtypes
    lib.orc_quad_cells_cos.restype = C.c_int
    return lib


def _cells(lib, ra, dec, r, L):
    buf = (C.c_uint64 * 5)()
    m = lib.orc_quad_cells(ra, dec, r, L, buf)
    return [int(buf[i]) for i in range(m)]


def test_unmutated_copy_reproduces_the_cases(tmp_path):
    lib = _build_mutant(tmp_path, "none", [])
    for ra, dec, r, L, want in CASES:
        assert _cells(lib, ra, dec, r, L) == want


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_misreading_fails_a_hand_placed_case(tmp_path, name):
    lib = _build_mutant(tmp_path, name, MUTANTS[name])
    wrong = [c[:4] for c in CASES if _cells(lib, *c[:4]) != c[4]]
    assert wrong, f"misreading {name} passes every hand-placed case"


# Misreadings of the variant's RA shift, checked against its own cases.
MUTANTS_COS = {
    "times_cos_not_over": [("double RA = c > 0.0 ? R / c : 180.0;",
                            "double RA = c > 0.0 ? R * c : 180.0;")],
    "no_cap_at_180": [("  if (RA > 180.0) RA = 180.0;\n  return RA;", "  return RA;")],
    "cos_of_radians": [("  orc_sincos_deg(dec, &sd, &cd);\n  double c = fabs(cd);",
                        "  orc_sincos_deg(dec, &sd, &cd);\n  double c = fabs(cos(dec));")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS_COS))
def test_each_misreading_of_the_variant_fails_a_case(tmp_path, name):
    lib = _build_mutant(tmp_path, name, MUTANTS_COS[name])
    buf = (C.c_uint64 * 5)()
    wrong = []
    for ra, dec, r, L, want in CASES_COS:
        m = lib.orc_quad_cells_cos(ra, dec, r, L, buf)
        if [int(buf[i]) for i in range(m)] != want:
            wrong.append((ra, dec))
    assert wrong, f"misreading {name} passes every hand-placed case of the variant"
