"""Filler cells (Section III-B) on the host: the oracle's rule against a
hand-worked example, and the library's fftpl_fillers against the oracle
(exact: the same double arithmetic rounded once to float32).

Hand example: region 10 x 10 (area 100); one fixed 4 x 4 cell centred at
(1, 1) overlaps the region on [0, 3] x [0, 3] (area 9), so the free area is
91; movable cells 1x1, 2x1, 3x2 (area 9, mean 2 x 4/3).  With rho_t = 0.5
the fillers take 0.5 * 91 - 9 = 36.5, each fl32(2) * fl32(4/3) =
2.6666667461..., so 13 fillers (36.5 / 2.66667 = 13.69).  With rho_t = 0.09
the movable cells already exceed 0.09 * 91 = 8.19: no fillers.
"""
import numpy as np
import pytest

import oracle
import synth


def hand():
    w = np.array([1, 2, 3, 4], np.float32)
    h = np.array([1, 1, 2, 4], np.float32)
    return dict(region=(0.0, 0.0, 10.0, 10.0), w=w, h=h, m_mov=3,
                fix_x=np.array([1.0], np.float32), fix_y=np.array([1.0], np.float32))


def test_oracle_rule_hand_example():
    cnt, fw, fh = oracle.fillers(**hand(), target_density=0.5)
    assert fw == 2.0 and fh == np.float32(4.0 / 3.0)
    assert cnt == 13
    cnt, _, _ = oracle.fillers(**hand(), target_density=0.09)
    assert cnt == 0


@pytest.fixture(scope="module")
def F():
    from paper_1312_4587_gb300 import _build
    _build.build()
    from paper_1312_4587_gb300 import fftpl
    fftpl.lib()
    return fftpl


@pytest.mark.parametrize("rho_t", [0.5, 0.09, 1.0])
def test_library_rule_matches_oracle_hand(F, rho_t):
    assert F.fftpl_fillers(**hand(), target_density=rho_t) == \
        oracle.fillers(**hand(), target_density=rho_t)


@pytest.mark.parametrize("name", ["tiny", "medium", "large"])
def test_library_rule_matches_oracle_instances(F, name):
    inst = synth.make_instance(name)
    args = dict(region=inst.region, w=inst.w, h=inst.h, m_mov=inst.m_mov, fix_x=inst.fix_x,
                fix_y=inst.fix_y, target_density=inst.target_density)
    got = F.fftpl_fillers(**args)
    assert got == oracle.fillers(**args)
    cnt, fw, fh = got
    # the fillers bring the movable area to rho_t of the free area (to within one filler)
    L = (inst.region[2] - inst.region[0]) * (inst.region[3] - inst.region[1])
    mov = float(np.dot(inst.w[:inst.m_mov].astype(np.float64), inst.h[:inst.m_mov]))
    fixed = float(np.dot(inst.w[inst.m_mov:].astype(np.float64), inst.h[inst.m_mov:]))
    target = inst.target_density * (L - fixed)
    assert target - fw * fh <= mov + cnt * fw * fh <= target + 1e-6 * target


def test_synth_appends_pinless_movable_cells():
    inst = synth.make_instance("medium")
    ext = synth.with_fillers(inst, 100, 2.0, 1.0)
    assert ext.m_mov == inst.m_mov + 100 and ext.m_fix == inst.m_fix
    assert np.all(ext.w[inst.m_mov:inst.m_mov + 100] == 2.0)
    np.testing.assert_array_equal(ext.w[ext.m_mov:], inst.w[inst.m_mov:])
    # pins keep their cells: movable ids unchanged, fixed ids shifted
    pc, opc = ext.pin_cell, inst.pin_cell
    np.testing.assert_array_equal(pc[opc < inst.m_mov], opc[opc < inst.m_mov])
    np.testing.assert_array_equal(pc[opc >= inst.m_mov], opc[opc >= inst.m_mov] + 100)
    assert not np.any((pc >= inst.m_mov) & (pc < ext.m_mov))   # fillers have no pins


def test_fillers_rejects_bad_arguments(F):
    bad = hand()
    bad["w"] = bad["w"].copy(); bad["w"][0] = -1.0
    with pytest.raises(F.FFTPLError) as ei:
        F.fftpl_fillers(**bad)
    assert ei.value.status == F.FFTPL_EINVAL
    with pytest.raises(F.FFTPLError):
        F.fftpl_fillers(**hand(), target_density=0.0)
