"""The C-ABI library loads (no GPU needed) and exports every function that
include/emm.h declares; host-side error paths return the documented codes."""
import os
import re

import numpy as np
import pytest

import paper_2304_00233_b300 as emm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(emm_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = emm.load_library()
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared == set(emm.EXPORTED), declared ^ set(emm.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_codes():
    for code in range(9):
        assert emm.strerror(code)
    assert emm.strerror(99) == "unknown error"


def test_grid_errors():
    x = np.arange(10.0)
    with pytest.raises(emm.EmmError) as e:
        emm.make_grid(x, x, x, rd=5)
    assert e.value.code == emm.EMM_EINVAL
    with pytest.raises(emm.EmmError):
        emm.make_grid(x[::-1], x, x, rd=2)           # not ascending
    with pytest.raises(emm.EmmError):
        emm.make_grid(x, x, x, rd=3, nb=2)          # nb < rd
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    assert g.npad == (24, 24, 24) and g.cells == 24 ** 3
    with pytest.raises(emm.EmmError) as e:
        g.locate(0, (-100.0, 4.0, 4.0))             # left of the grid
    assert e.value.code == emm.EMM_EOUTSIDE
    with pytest.raises(emm.EmmError) as e:
        g.locate(0, (-4.5, 4.0, 4.0))               # inside the pads but in the CPML
    assert e.value.code == emm.EMM_EOUTSIDE
    g.locate(0, (4.2, 4.0, 4.0))


def test_survey_errors_before_any_device_call():
    x = np.arange(12.0) * 10
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    good = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(55, 55, 55),
                      rec=np.array([[40.0, 50.0, 60.0]]), freqs=[1.0])
    assert emm.workspace_size(g, good) > 0
    for bad in (dict(omega0=0.0), dict(fmax=-1.0), dict(sigma_min=0.0), dict(nt=-1), dict(freqs=[]),
                dict(src_kind=2), dict(src_length=-1.0), dict(src_length=100.0, src_points=0),
                dict(src_length=100.0, src_points=257)):
        s = emm.Survey(**{**good.__dict__, **bad})
        with pytest.raises(emm.EmmError) as e:
            emm.workspace_size(g, s)
        assert e.value.code == emm.EMM_EINVAL


def test_antenna_workspace_holds_the_union_boxes():
    # an antenna's weights need more room than a point dipole's (2rd)^3 boxes
    x = np.arange(40.0) * 10
    g = emm.make_grid(x, x, x, rd=2, nb=4, ne=3)
    point = emm.Survey(omega0=1.0, fmax=1.0, sigma_min=1.0, nt=10, src=(195, 195, 195),
                       rec=np.array([[150.0, 150.0, 150.0]]), freqs=[1.0])
    ant = emm.Survey(**{**point.__dict__, "src_length": 60.0, "src_points": 6})
    assert emm.workspace_size(g, ant) > emm.workspace_size(g, point)

