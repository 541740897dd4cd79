"""Workload configurations as JSON (CPU only).

The five benchmark configurations ship as JSON files beside the workload
module; each must describe exactly the workload the tests and the benchmark
build from the module's constants, and round-trip through to_dict/from_dict.
"""
import json
import os

import pytest

from paper_1909_13412_gb300 import workloads as wl

CONFIGS = {
    "config1_relaxation_32.json": wl.RELAXATION_32,
    "config2_brownian_128.json": wl.BROWNIAN_128,
    "config3_brownian_256.json": wl.BROWNIAN_256,
    "config4_ensemble_68.json": wl.ENSEMBLE_68,
    "config5_adjoint_64.json": wl.ADJOINT_64,
}


@pytest.mark.parametrize("fname", sorted(CONFIGS))
def test_config_files_describe_the_benchmark_workloads(fname):
    w = wl.load(os.path.join(wl.CONFIG_DIR, fname))
    assert w == CONFIGS[fname]
    assert w.nodes == CONFIGS[fname].nodes
    assert wl.from_dict(json.loads(json.dumps(wl.to_dict(w)))) == w


def test_every_config_file_is_listed():
    assert sorted(f for f in os.listdir(wl.CONFIG_DIR) if f.endswith(".json")) == sorted(CONFIGS)


def test_unknown_kind_and_fields_are_refused():
    with pytest.raises(ValueError):
        wl.from_dict({"kind": "torus", "name": "x"})
    with pytest.raises(TypeError):
        wl.from_dict({"kind": "box", "name": "x", "shape_zyx": [4, 4, 4], "tau": 0.8, "n_particles": 1,
                      "viscosity": 0.1})
