"""The roofline formulas reproduce the numbers the paper prints (Sec. 3, 3.3, Table 'alpha values')."""
import json
import os

import pytest

from paper_1907_06487_gb300 import perfmodel as pm

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_roofline.json")))


def test_spin26_alpha_from_measured_bytes():
    s = G["spin26"]
    a = pm.alpha_from_spmv_bytes(s["bytes_per_nnz_ivb"], s["nnzr"])
    assert round(a, 3) == s["alpha_ivb"]


def test_spin26_symm_bounds():
    s = G["spin26"]
    a_ivb = pm.alpha_from_spmv_bytes(s["bytes_per_nnz_ivb"], s["nnzr"])
    i_ivb = pm.i_symm_spmv(a_ivb, s["nnzr"])
    assert abs(pm.perf(i_ivb, s["bw_ivb_copy"]) - s["perf_ivb"][0]) <= 0.01
    assert abs(pm.perf(i_ivb, s["bw_ivb_load"]) - s["perf_ivb"][1]) <= 0.01
    i_skx = pm.i_symm_spmv(s["alpha_skx"], s["nnzr"])
    assert abs(pm.perf(i_skx, s["bw_skx_copy"]) - s["perf_skx"][0]) <= 0.01
    assert abs(pm.perf(i_skx, s["bw_skx_load"]) - s["perf_skx"][1]) <= 0.01


@pytest.mark.parametrize("row", G["alpha_table"]["rows"], ids=lambda r: r["matrix"])
def test_alpha_table(row):
    nnzr = row["nnzr"]
    if row["matrix"] in G["exact_nnzr"]:
        nnz, nr = G["exact_nnzr"][row["matrix"]]
        nnzr = nnz / nr
    assert 1.0 / nnzr == pytest.approx(row["alpha_opt"], rel=1e-7)
    assert pm.i_spmv(1.0 / nnzr, nnzr) == pytest.approx(row["i_spmv"], rel=1e-7)
    if "alpha_symm_opt" in row:
        assert 1.0 / pm.nnzr_symm(nnzr) == pytest.approx(row["alpha_symm_opt"], rel=1e-7)


def test_gpu_traffic_figures():
    # XXZ L=26 periodic: N = 10,400,600; nnz_u = 80,708,656; nnz_f = 151,016,712
    n, nu, nf = 10400600, 80708656, 151016712
    assert nf == 2 * nu - n
    assert pm.symm_bytes(n, nu) == 12 * nu + 4 * (n + 1) + 16 * n
    assert pm.full_bytes(n, nf) == 12 * nf + 4 * (n + 1) + 16 * n
    assert pm.flops(nf) == 302033424
    assert pm.symm_bytes(n, nu, val_bytes=4) == pm.symm_bytes(n, nu) - 4 * nu


def test_accumulate_byte_count_is_the_papers_intensity_at_optimal_alpha():
    """symm_bytes_rmw equals the bytes of Eq. SymmSpMV_intensity at
    alpha = 1 / N_nzr^symm (4 flops per stored nonzero over the intensity),
    on the XXZ L=26 and 27-point 200^3 sizes."""
    for n, nu in ((10400600, 80708656), (8000000, 110923596)):
        nsym = nu / n
        nnzr = 2.0 * (nsym - 1.0) + 1.0  # inverse of Eq. NNZR_symm
        paper = nu * 4.0 / pm.i_symm_spmv(1.0 / nsym, nnzr)
        assert pm.symm_bytes_rmw(n, nu) == pytest.approx(paper, rel=1e-12)
        assert pm.symm_bytes_rmw(n, nu) - pm.symm_bytes(n, nu) == 8 * n - 4
