"""The byte model bench.py reports (host logic, CPU): the per-pass table adds
up to the iteration totals the roofline fractions are quoted on."""
import bench


def iotf_passes():
    return (["col_q", "row_mul_t", "col_q", "row_intensity", "col_resid_iotf2", "row_mul_v", "col_q",
             "row_mul_t", "col_q", "row_grad_pack", "col_precond_reg", "row_nesterov_fft"])


def modal_passes(k):
    fwd = ["col_mode_fwd", "row_mul_t", "col_q", "row_mode_int"]
    back = ["row_mode_vg", "col_q", "row_mul_t", "col_mode_back"]
    return (["col_fft"] + fwd * k + ["modal_resid"] + back * k + ["col_ifft", "row_grad_pack", "col_precond_reg",
                                                                     "row_nesterov_fft"])


def iotf_packed_passes():
    p = iotf_passes()
    i = p.index("row_intensity")
    p[i:i + 3] = ["row_intensity_pk", "col_resid_pk", "row_mul_v_pk"]
    return p


def test_iotf_iteration_is_296_bytes_per_pixel():
    assert sum(bench.PASS_BYTES_PER_PX[p] for p in iotf_passes()) == 296


def test_packed_residual_saves_20_bytes_per_pixel():
    # packed F_row{|v|^2} and residual: 4 B/px each way instead of 8; the
    # column pass reads F{y} of bins 0..nx/2 only
    assert sum(bench.PASS_BYTES_PER_PX[p] for p in iotf_packed_passes()) == 276


def test_modal_iteration_matches_the_closed_form():
    for k in (1, 9, 25):
        assert sum(bench.PASS_BYTES_PER_PX[p] for p in modal_passes(k)) == bench.modal_bytes_per_px(k)
    assert bench.modal_bytes_per_px(9) == 1632 and bench.modal_bytes_per_px(25) == 4256


def test_state_floor_is_what_an_iteration_must_touch():
    # psi read and written, phi read and written, t and y read
    assert bench.STATE_FLOOR_BYTES_PER_PX == 8 + 8 + 8 + 8 + 8 + 4


def test_issue_roofline_arithmetic():
    # 32 thread instructions per pixel over 1 Gpx in 1 s: 1 G warp-instructions/s;
    # 100 SMs x 4 schedulers at 1000 MHz issue 400 G warp-instructions/s
    r = bench.issue_roofline(32.0, 1e9, 1000.0, 100, 1000.0)
    assert abs(r["achieved"] - 1.0) < 1e-12 and abs(r["peak"] - 400.0) < 1e-9
    assert abs(r["frac"] - 1.0 / 400.0) < 1e-15


def test_instruction_count_only_for_the_captured_sources(monkeypatch):
    ipx = bench.measured_instructions_per_px("col_q")
    if ipx is not None:  # the committed capture matches the current kernel sources
        assert 50 < ipx < 200
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.measured_instructions_per_px("col_q") is None
    assert bench.measured_traffic("col_q") is None


def test_selected_shape_ids_parse_the_plan_description():
    import bench
    d = ("ny=1024 nx=1024 batch=180 solver=graph loop=none col_q=C8s2[C8p:0.98,C8s2:0.88,C8s2@8.8.16:0.90] "
         "col_iotf=C8s2@8.8.16[C8p:0.92,C8s2:0.87,C8s2@8.8.16:0.85] col_fft=C8p "
         "col_resid_pk=C16s2@8.8.16[C8s2:0.74,C16s2:0.71,C16s2@8.8.16:0.70]")
    assert bench.selected_shape_ids(d) == [1, 2, None, 2]
