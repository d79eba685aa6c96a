"""Host side of the launch-shape autotuner: the table API and the VD_TUNE_FILE round trip.

Runs without a GPU: setting and listing entries, and reading the file at the first query of
a fresh process, are host computations.
"""

import os
import subprocess
import sys
import textwrap

import pytest

import paper_2403_06654_gb300 as vd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_set_list_erase():
    vd.vd_autotune_set(0, 1, 96, 2, -1, 8)
    vd.vd_autotune_set(1, 2, 48, 0, 0, 4)
    tab = vd.vd_autotune_table()
    assert (0, 1, 96, 2, -1, 8) in tab and (1, 2, 48, 0, 0, 4) in tab
    vd.vd_autotune_set(0, 1, 96, 2, -1, -1)
    assert (0, 1, 96, 2, -1, 8) not in vd.vd_autotune_table()


@pytest.mark.parametrize("bad", [(2, 0, 64, 1, 1, 4), (0, 3, 64, 1, 1, 4), (0, 0, 0, 1, 1, 4),
                                 (0, 0, 64, 1, 1, 3), (0, 0, 64, 1, 1, 256), (0, 0, 64, 1, 1, 96)])
def test_bad_keys_rejected(bad):
    with pytest.raises(vd.VDError) as e:
        vd.vd_autotune_set(*bad)
    assert e.value.status == vd.VD_ERR_INVALID_ARG


def test_staged_choice_accepted():
    """Choice 128 selects the TMA-staged kernels (float y/z passes, fused x pass)."""
    vd.vd_autotune_set(0, 1, 256, 2, 1, 128)
    assert (0, 1, 256, 2, 1, 128) in vd.vd_autotune_table()
    vd.vd_autotune_set(0, 1, 256, 2, 1, -1)


def test_file_read_by_a_fresh_process(tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("0 1 256 2 -1 0\n1 0 80 0 2 16\n0 2 160 1 1 4\n")
    code = textwrap.dedent("""
        import paper_2403_06654_gb300 as vd
        print(sorted(vd.vd_autotune_table()))
    """)
    env = dict(os.environ, VD_TUNE_FILE=str(f), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True).stdout
    assert out.strip() == str(sorted([(0, 1, 256, 2, -1, 0), (1, 0, 80, 0, 2, 16), (0, 2, 160, 1, 1, 4)]))
