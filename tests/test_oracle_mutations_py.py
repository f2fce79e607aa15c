"""Plausible mistakes planted in copies of the Python oracles (smoothness
loss, Adam step, LiDAR targets and loss) must each fail one of their pins.

Each case rewrites one line of the oracle's source in memory, loads the copy
as a separate module, points the `oracle` package's names at the copy's
functions, and runs every pin of that oracle's test file; at least one pin
has to fail.  Nothing on disk changes.  CPU only.
"""
import importlib
import inspect
import os
import types

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle module, pin test module, names exported by the oracle package, old, new)
MUTATIONS = {
    "smooth_diagonal_neighbour": (
        "smooth", "test_oracle_smooth", ("neighbour_ids", "smooth_loss"),
        "NEIGHBOURS = ((-1, 0), (1, 0), (0, -1), (0, 1))",
        "NEIGHBOURS = ((-1, -1), (1, 0), (0, -1), (0, 1))"),
    "smooth_offroad_is_surfel_0": (
        "smooth", "test_oracle_smooth", ("neighbour_ids", "smooth_loss"),
        "out[ids, k] = np.where(nb >= 0, nb, ids)",
        "out[ids, k] = np.where(nb >= 0, nb, 0)"),
    "smooth_wrong_normalisation": (
        "smooth", "test_oracle_smooth", ("neighbour_ids", "smooth_loss"),
        "L = float(np.sum(d * d)) / K",
        "L = float(np.sum(d * d)) / (2 * K)"),
    "smooth_neighbour_gradient_sign": (
        "smooth", "test_oracle_smooth", ("neighbour_ids", "smooth_loss"),
        "np.add.at(g, j, -2.0 * d / K)",
        "np.add.at(g, j, 2.0 * d / K)"),
    "smooth_neighbour_gradient_dropped": (
        "smooth", "test_oracle_smooth", ("neighbour_ids", "smooth_loss"),
        "np.add.at(g, j, -2.0 * d / K)",
        "pass"),
    "adam_no_bias_correction": (
        "adam", "test_oracle_adam", ("adam_step", "z_learning_rate"),
        "mh = m / (1.0 - b1 ** t)",
        "mh = m"),
    "adam_eps_inside_sqrt": (
        "adam", "test_oracle_adam", ("adam_step", "z_learning_rate"),
        "return p - lr * mh / (np.sqrt(vh) + eps), m, v",
        "return p - lr * mh / np.sqrt(vh + eps), m, v"),
    "adam_beta2_in_first_moment": (
        "adam", "test_oracle_adam", ("adam_step", "z_learning_rate"),
        "m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g",
        "m = b2 * np.asarray(m, np.float64) + (1.0 - b2) * g"),
    "adam_z_rate_linear_decay": (
        "adam", "test_oracle_adam", ("adam_step", "z_learning_rate"),
        "return scene_size * start * (end / start) ** f",
        "return scene_size * (start + (end - start) * f)"),
    "lidar_radius_not_squared": (
        "lidar", "test_oracle_lidar", ("nearest_elevation", "elev_loss"),
        "ok = dmin <= radius * radius",
        "ok = dmin <= radius"),
    "lidar_ties_take_highest_index": (
        "lidar", "test_oracle_lidar", ("nearest_elevation", "elev_loss"),
        "j = np.argmin(d2, axis=1)",
        "j = d2.shape[1] - 1 - np.argmin(d2[:, ::-1], axis=1)"),
    "lidar_gradient_factor": (
        "lidar", "test_oracle_lidar", ("nearest_elevation", "elev_loss"),
        "return float(np.sum(d * d)), 2.0 * d",
        "return float(np.sum(d * d)), d"),
    "lidar_untargeted_surfels_count": (
        "lidar", "test_oracle_lidar", ("nearest_elevation", "elev_loss"),
        "d = np.where(has, z - np.where(has, zbar, 0.0), 0.0)",
        "d = np.where(has, z - np.where(has, zbar, 0.0), z)"),
}


def mutated_module(name, old, new):
    path = os.path.join(ROOT, "oracle", name + ".py")
    src = open(path).read()
    assert src.count(old) == 1, (name, old)
    mod = types.ModuleType("oracle_mutant_" + name)
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    return mod


def run_pins(test_module):
    """Number of pins of `test_module` that fail (skipped pins do not count)."""
    tm = importlib.import_module(test_module)
    failed = 0
    for fname, fn in inspect.getmembers(tm, inspect.isfunction):
        if not fname.startswith("test_") or inspect.signature(fn).parameters:
            continue
        try:
            fn()
        except pytest.skip.Exception:
            continue
        except Exception:   # an assertion or an error both mean the pin caught it
            failed += 1
    return failed


def test_pins_pass_on_the_oracle_as_it_stands():
    for test_module in ("test_oracle_smooth", "test_oracle_adam", "test_oracle_lidar"):
        assert run_pins(test_module) == 0, test_module


@pytest.mark.parametrize("case", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    name, test_module, exported, old, new = MUTATIONS[case]
    mod = mutated_module(name, old, new)
    for attr in exported:
        monkeypatch.setattr(oracle, attr, getattr(mod, attr))
    assert run_pins(test_module) >= 1, case
