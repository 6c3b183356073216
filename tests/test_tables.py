"""The coefficient tables shipped in paper_2605_08523_gb300/tables (written by
the library's GPU trainer, paper_2605_08523_gb300.train_tables): metadata, and
their fit error re-measured with the oracle's scalar recursion against the
target functions (the tables are outputs under test; the expected values are
the logistic and entropy definitions).  CPU only."""
import glob
import json
import os

import numpy as np
import pytest

from oracle import altform, maxsp2, skipsp2, tables, train

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(glob.glob(os.path.join(ROOT, "paper_2605_08523_gb300", "tables", "*.json")))


def load(name):
    with open(os.path.join(ROOT, "paper_2605_08523_gb300", "tables", name + ".json")) as f:
        return json.load(f)


def test_tables_present():
    names = {os.path.basename(f)[:-5] for f in FILES}
    assert "entropy_b1500_L26" in names
    for b in (20, 50, 100, 200):
        for L in (16, 24, 32):
            assert "b%d_L%d" % (b, L) in names


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_table_fit_errors(path):
    d = json.load(open(path))
    b0, m0, al = d["beta0"], d["mu0"], d["alpha"]
    if "max" in d:
        # Max-SP2 (flat table; Skip-SP2 (k, K) tables carry their Max-SP2 embedding)
        p, pe = np.array(d["max"]), np.array(d["max_entropy"])
        assert p.size == maxsp2.nparams(d["L"]) and pe.size == maxsp2.nparams(d["L"])
        if "skipk" in d:
            # the stored embedding is that of the stored Skip-SP2 vector
            k, K, L = d["k"], d["K"], d["L"]
            t = maxsp2.skip_unpack(np.array(d["skipk"]), L, k, K)
            assert np.max(np.abs(maxsp2.skip_to_max(t) - p)) < 1e-12 * max(1.0, np.max(np.abs(p)))
        ef = maxsp2.max_error(p, d["L"], "fermi", b0, m0, 1.0, grid=400001)
        es = maxsp2.max_error(pe, d["L"], "entropy", b0, m0, al, grid=400001)
    elif "skip" in d:
        # Skip-SP2 (one stored layer, one accumulator): the oracle's recursion of that family
        t, te = np.array(d["skip"]), np.array(d["skip_entropy"])
        assert t.shape == (d["L"] + 1, 4) and te.shape == (d["L"] + 1, 4)
        ef = skipsp2.max_error(t, "fermi", b0, m0, 1.0, grid=400001)
        es = skipsp2.max_error(te, "entropy", b0, m0, al, grid=400001)
    elif "alt" in d:
        # one-term form (Eq. mlsp2_alt): evaluated with the oracle's own recursion of that form
        a, ae = np.array(d["alt"]), np.array(d["alt_entropy"])
        assert a.shape == (d["L"] + 1, 2) and ae.shape == (d["L"] + 1, 2)
        ef = altform.max_error(a, "fermi", b0, m0, 1.0, grid=400001)
        es = altform.max_error(ae, "entropy", b0, m0, al, grid=400001)
    else:
        th = np.array(d["theta"])
        ths = np.array(d["theta_entropy"])
        assert th.shape == (d["L"], 4) and ths.shape == (d["L"], 4)
        ef = train.max_error(th, "fermi", b0, m0, 1.0, grid=400001)
        es = train.max_error(ths, "entropy", b0, m0, al, grid=400001)
    # the recorded GPU figures agree with the oracle's evaluation
    assert ef == pytest.approx(d["fit"]["max_err_fermi"], rel=0.05, abs=1e-9)
    assert es == pytest.approx(d["fit"]["max_err_entropy"], rel=0.05, abs=1e-9)


def test_entropy_table_for_printed_weights():
    d = load("entropy_b1500_L26")
    assert np.array_equal(np.array(d["theta"]), np.array(tables.PRINTED_B1500))
    es = train.max_error(np.array(d["theta_entropy"]), "entropy", 1500.0, 1 / 3, 0.842704, grid=2_000_001)
    e_fermi = train.max_error(np.array(d["theta"]), "entropy", 1500.0, 1 / 3, 0.842704, grid=2_000_001)
    # Table entropy: theta_fermi 1.24e-3; training theta_entropy improves it by orders of magnitude
    assert abs(e_fermi - 1.24e-3) < 1e-5
    assert es < 1e-6


def test_one_term_tables():
    # trained in the one-term form from the SP2 sequence; the fit reaches ~1e-5
    for name in ("alt_b1500_L26", "alt_b100_L16"):
        d = load(name)
        assert d["fit"]["max_err_fermi"] < 3e-5 and d["fit"]["max_err_entropy"] < 3e-5, name


def test_skip_tables():
    # the accumulator feedback improves the embedded printed table's fit
    d = load("skip_b1500_L26")
    assert d["fit"]["max_err_fermi"] < 0.5 * d["fit"]["max_err_fermi_start"]
    assert d["fit"]["max_err_fermi"] < 1e-7 and d["fit"]["max_err_entropy"] < 1e-5
    assert max(abs(r[2]) for r in d["skip"][:-1]) > 0.0
    assert load("skip_b100_L16")["fit"]["max_err_fermi"] < 3e-5


def test_training_sweep_layer_count():
    # Eq. layer count: beta0 = 200 needs n_l = 18.5 layers, so 16 layers
    # underfit while 24 and 32 reach ~1e-6; every trained table beats its SP2
    # initial guess by orders of magnitude (what the learned part gains).
    e = {(b, L): load("b%d_L%d" % (b, L))["fit"] for b in (20, 50, 100, 200) for L in (16, 24, 32)}
    assert e[(200, 16)]["max_err_fermi"] > 5 * e[(200, 24)]["max_err_fermi"]
    for k, f in e.items():
        assert f["max_err_fermi"] < 1e-3 * f["max_err_sp2_init"], k
        assert f["max_err_fermi"] < 3e-5, k


def test_family_tables_layers_saved():
    # beta0 = 100: the 12-layer Max-SP2 table fits as well as the 14-layer
    # Eq. mlsp2 table; at 10 layers Max-SP2 is far ahead of Eq. mlsp2 and
    # Skip-SP2 (2, 2) sits between them
    e = {n: load(n)["fit"]["max_err_fermi"] for n in ("b100_L10", "b100_L12", "b100_L14", "max_b100_L10",
                                                       "max_b100_L12", "skip22_b100_L10", "skip22_b100_L12")}
    assert e["max_b100_L12"] < e["b100_L14"]
    assert e["max_b100_L10"] < 0.1 * e["b100_L10"] and e["max_b100_L10"] < e["b100_L12"]
    assert e["max_b100_L10"] < e["skip22_b100_L10"] < e["b100_L10"]
    assert e["skip22_b100_L12"] < e["b100_L12"]


def test_grid_command_line():
    # the command lines that produced the polished tables
    from paper_2605_08523_gb300.train_tables import grid_args
    assert grid_args(["x", "OUT", "--grid", "2250:27", "5000", "--polish", "14"]) == ("OUT", [(2250.0, 27)], 5000, 14)
    assert grid_args(["x", "OUT", "--grid", "100:18,200:21", "5000", "--polish", "6"]) == \
        ("OUT", [(100.0, 18), (200.0, 21)], 5000, 6)
    assert grid_args(["x", "--polish", "6", "OUT", "--grid", "400:24"]) == ("OUT", [(400.0, 24)], 3000, 6)
    assert grid_args(["x", "OUT", "--grid", "2250:32"]) == ("OUT", [(2250.0, 32)], 3000, 0)


def test_polished_tables_record_their_passes():
    for name in ("b2250_L27", "b100_L18", "b200_L21", "b400_L24"):
        d = load(name)
        assert d["train"]["fermi"]["polish_passes"] >= 6 and 0 <= d["train"]["fermi"]["kept_pass"] <= \
            d["train"]["fermi"]["polish_passes"], name


def test_bench_model_sets_exist():
    # every table the bench's workloads load is shipped and carries its fit
    import types
    import bench
    sets = [bench.ragged_table_paths()]
    for wk, kT in (("longrange", 0.1), ("lattice", 0.1), ("lattice", 0.05), ("lattice", 0.3)):
        sets.append(bench.table_paths(types.SimpleNamespace(workload=wk, kT=kT, table="printed")))
    for tb in ("skip", "alt"):
        sets.append(bench.table_paths(types.SimpleNamespace(workload="lattice", kT=0.1, table=tb)))
    sets.append([os.path.join(bench.TABLE_DIR, nm + ".json") for nm in bench.FAMILY_TABLES])
    for paths in sets:
        assert paths
        for p in paths:
            assert os.path.exists(p), p
            d = json.load(open(p))
            assert "fit" in d or os.path.basename(p) == "entropy_b1500_L26.json", p
