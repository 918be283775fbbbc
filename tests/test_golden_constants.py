"""The constants the paper prints (tests/golden/paper_constants.txt, each with its citation) are the
ones the oracle and the CUDA path use.  CPU only: the GPU side is read from the library's host
function mgfld_eos_default and from the kernel header's text."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from oracle import mgfld_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _golden():
    out = {}
    for line in open(os.path.join(HERE, 'golden', 'paper_constants.txt')):
        line = line.strip()
        if not line or line.startswith('#'):
            continue
        name, value, cite = line.split(None, 2)
        assert cite.startswith(('Eq.', 'Sec.', 'text')), name
        out[name] = float(Fraction(value))
    return out


def _header():
    return open(os.path.join(ROOT, 'paper_1809_05608_gb300', 'csrc', 'mgfld_internal.cuh')).read()


def test_oracle_uses_the_printed_constants():
    g = _golden()
    p = O.EosParams()
    assert p.gamma1 == g['gamma1'] and p.g_n == g['g_n'] and p.g_p == g['g_p']
    assert list(O.STAT_WEIGHT) == [g['stat_weight_nue'], g['stat_weight_nuebar'], g['stat_weight_numt'],
                                   g['stat_weight_numtbar']]
    assert O.SHOCK_ROLL_IN == (g['shock_roll_in_start'], g['shock_roll_in_full'])
    # Eq. e6 at the printed proton fraction: the cold pressures agree at rho_nuc
    n = g['x_p_for_f2'] * p.rho_nuc / p.m_b
    p1 = (p.gamma1 - 1) * p.f1 * n ** p.gamma1
    p2 = (p.gamma2 - 1) * p.f2 * n ** p.gamma2
    assert abs(p1 / p2 - 1) < 1e-13


def test_cuda_path_uses_the_printed_constants():
    g = _golden()
    src = _header()
    m = re.search(r'constexpr double kShockOn = ([0-9.eE+-]+), kShockFull = ([0-9.eE+-]+);', src)
    assert m and (float(m.group(1)), float(m.group(2))) == (g['shock_roll_in_start'], g['shock_roll_in_full'])
    m = re.search(r'stat_weight\(int q\) \{ return q < 2 \? ([0-9.]+) : ([0-9.]+); \}', src)
    assert m and (float(m.group(1)), float(m.group(2))) == (g['stat_weight_nue'], g['stat_weight_numt'])
    assert g['stat_weight_nuebar'] == g['stat_weight_nue'] and g['stat_weight_numtbar'] == g['stat_weight_numt']
    from paper_1809_05608_gb300 import mgfld as M
    if not os.path.exists(M.LIB_PATH):
        pytest.skip('library not built')
    e = M.lib().mgfld_eos_default()
    assert e.gamma1 == g['gamma1'] and e.g_n == g['g_n'] and e.g_p == g['g_p']
    assert e.rho_nuc == O.EosParams().rho_nuc            # reading of the EoS section, the same on both sides
