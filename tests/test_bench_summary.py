"""The compact variant summary bench.py appends as the JSON line's last key: the
headline figures of the variants it names, rounded, and nothing for variants
that did not run (CPU, no GPU needed)."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_summary_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _gain(speedup, fallback, uerr):
    return {"speedup": speedup, "fallback_rate": fallback, "u_error_after_4_advances_vs_lbm": uerr,
            "u_error_at_horizon_vs_lbm": 2 * uerr}


def test_summary_rounds_the_named_figures():
    variants = {
        "kh2048_f16dev": {"mlups": 60211.4, "speedup_vs_f32": 1.76612},
        "kh2048_bf16dev": {"mlups": 60144.6},
        "kh2048_f64": {"mlups": 2564.4},
        "kh2047_f32_plain_layout": {"mlups": 33472.5},
        "kh2048_f32_4slabs": {"mlups": 30279.7},
        "kh2048_f32_diagnostics_every_10": {"overhead": 0.04866},
        "kh3d256_d3q125_f32": {"mlups": 6310.6, "frac_of_measured_hbm": 0.93183},
        "kh3d256_d3q125_f16dev": {"mlups": 10403.6, "frac_of_measured_hbm": 0.76811},
        "kh3d256_d3q125_bf16dev": {"mlups": 10502.3, "frac_of_measured_hbm": 0.77539},
        "batched_256_f32": {"persistent_graph": {"mlups": 30130.2, "gbs_algorithmic": 6026.0},
                            "speedup_persistent_graph_vs_per_instance": 1.2662},
        "surrogate_kh256": {"gain_test": {"by_tol": {"1e-4": _gain(0.888, 0.741, 0.0093),
                                                     "no gate": _gain(2.508, 0.0, 0.0671)}},
                            "speed_one_advance": {"64": {"speedup_vs_lbm": 2.5302}},
                            "training": {"tflops": 758.61}, "test_mse_normalised": {"network": 0.43931}},
    }
    out = _bench().variant_summary(variants, 6772.2)
    assert out["f16dev_mlups"] == 60211 and out["bf16dev_mlups"] == 60145 and out["f16dev_vs_f32"] == 1.77
    assert out["d3q125_256_f16dev_frac"] == 0.768 and out["diag_every10_overhead"] == 0.049
    assert out["batched_mlups"] == 30130 and out["batched_frac"] == round(6026.0 / 6772.2, 3)
    assert out["batched_vs_per_instance"] == 1.27
    assert out["surrogate_gain_speedup_fallback_uerr4"] == {"1e-4": [0.89, 0.74, 0.009], "no gate": [2.51, 0.0, 0.067]}
    assert out["surrogate_advance_speedup_b64"] == 2.53 and out["surrogate_heldout_mse"] == 0.439
    assert len(json.dumps(out)) < 1000   # stays within the end of the line a reader keeps


def test_summary_skips_what_did_not_run():
    bench = _bench()
    assert bench.variant_summary({}, 6772.2) == {}
    out = bench.variant_summary({"kh2048_f16dev": {"mlups": 1.0, "status": "ok"}, "batched_256_f32": {}}, 6772.2)
    assert out == {"f16dev_mlups": 1}
