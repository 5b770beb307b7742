"""The reference arm of bench.py (the oracle timed on all host cores, one
replica per core) prints one JSON line with the keys of the bench contract,
on the main arm's metric, naming the sample it ran (no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference', '--steps', '1',
                        '--warmup', '0'], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith('{')]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ('metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step', 'higher_is_better',
                'scaling', 'vs_baseline', 'dtype', 'data', 'config', 'impl', 'cpu_baseline', 'e2e'):
        assert key in line, key
    assert line['impl'] == 'reference' and line['n_gpus'] == 1 and line['steps'] == 1 and line['warmup'] == 0
    assert line['higher_is_better'] is True and line['vs_baseline'] is None and line['data'] == 'synthetic'
    assert line['value'] > 0 and line['unit'] == 'cell-updates/s'
    # the workload names what ran (the oracle on a 16^3-base sample), and what it samples
    assert line['config']['workload'].startswith('blast3d base 16x16x16, 3 levels, 16^3 patches, FP64, plain flags')
    assert line['config']['sample_of'].startswith('blast3d base 128x128x128, 3 levels, 16^3 patches')
    assert line['config']['leaf_cell_updates_per_s'] > 0
    cb = line['cpu_baseline']
    assert cb['kind'] == 'oracle' and cb['cores'] >= 1 and cb['value'] == line['value'] and cb['sample']
    e2e = line['e2e']
    assert e2e['value'] == line['value'] and e2e['unit'] == line['unit']
    assert e2e['h2d_bytes_per_step'] == 0 and e2e['d2h_bytes_per_step'] == 0


def test_set_tuning_parsing():
    """--set-tuning pins launch parameters by name (amr.TUNE_NAMES)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2508_05020_gb300.amr import TUNE_NAMES
    got = bench.parse_tuning('rhs_tile_shape=2, rhs_ctas_per_sm=1,')
    assert got == {'rhs_tile_shape': 2, 'rhs_ctas_per_sm': 1}
    assert set(got) <= set(TUNE_NAMES)
    assert bench.parse_tuning('') == {}
    for bad in ('rhs_tile_shape', '=2', 'rhs_tile_shape=two'):
        with pytest.raises(ValueError):
            bench.parse_tuning(bad)
