"""The synthetic workloads against the paper's own parameter table and task setup
(tests/golden/sim_params.txt: App. B, Table "sim_params", and App. B.1)."""
from pathlib import Path

import numpy as np
import pytest

from paper_2606_04206_gb300 import inputs

GOLDEN = Path(__file__).parent / "golden" / "sim_params.txt"


def table():
    rows, setup = {}, {}
    for line in GOLDEN.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if len(f) == 2:
            setup[f[0]] = float(f[1])
            continue
        num = lambda s: 0.0 if s == "--" else float(s)     # "--": no value (no such energy)
        rows.setdefault(f[0], []).append(dict(nv=int(f[1]), K=num(f[2]), E=num(f[3]), G=num(f[4]),
                                              inext=f[5] == "1", plastic=f[6] == "1"))
    return rows, setup


def check_rod(p, b, row):
    assert bool(p.inextensible[b]) == row["inext"]
    assert bool(p.plastic[b]) == row["plastic"]
    assert p.E[b] == pytest.approx(row["E"])
    assert p.G[b] == pytest.approx(row["G"])
    if not row["inext"]:
        assert p.K[b] == pytest.approx(row["K"])


def test_trajopt_materials_are_the_table_rows():
    rows, setup = table()
    p = inputs.trajopt(n_rods=12, frames=4)
    for b in range(12):
        row = {0: rows["Wiring-post"][0], 1: rows["Unknotting"][0], 2: rows["Letter-Art"][0]}[b % 3]
        check_rod(p, b, row)
    assert p.dt == pytest.approx(setup["frame_time"])
    assert p.substeps_min == int(setup["substeps"])
    assert inputs.trajopt.__defaults__[1] == int(setup["frames"])


def test_diff_materials_are_the_table_rows():
    rows, _ = table()
    p = inputs.diff(n_rods=8, frames=4)
    for b in range(8):
        check_rod(p, b, rows["Letter-Art"][0] if p.plastic[b] else rows["Unknotting"][0])


@pytest.mark.parametrize("make", [lambda: inputs.trajopt(n_rods=24, frames=2),
                                  lambda: inputs.batching(n_rods=24, frames=2),
                                  lambda: inputs.diff(n_rods=24, frames=2)])
def test_open_rods_are_smooth_and_rest_on_the_table(make):
    p = make()
    for b in range(p.batch):
        x = p.x_rest[p.vert_off[b]:p.vert_off[b + 1]]
        assert x[:, 2].min() == pytest.approx(0.005, abs=1e-6)     # just above the plane z = 0
        assert inputs._max_curvature(x) <= 50.0 + 1e-3               # bending radius >= 2 cm
