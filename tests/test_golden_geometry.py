"""The paper's printed geometry pins two readings used by every workload:
lambda_m is the mean of the (evenly spaced) band and the pitch is half the
shortest wavelength; the printed layer, FOV and detector-pixel sizes in units
of lambda_m then follow (FOV = 200 features, detector pixel = 8 features)."""
import os

import numpy as np

from paper_2604_02624_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_geometry.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = [float(t) for t in v.split(",")] if "," in v else float(v)
    return out


def test_lambda_m_is_band_mean_and_pitch_half_shortest():
    g = _golden()
    lam = np.linspace(g["lambda_longest_nm"], g["lambda_shortest_nm"], int(g["n_lambda"]))
    lam_m = lam.mean()
    assert abs(0.5 * lam.min() - g["pitch_nm"]) < 1e-9
    side = g["features_per_side"] * g["pitch_nm"] / lam_m
    assert abs(side - g["layer_side_in_lambda_m"]) < 0.5
    fov_features = g["fov_side_in_lambda_m"] * lam_m / g["pitch_nm"]
    assert abs(fov_features - 200) < 0.05
    px_features = g["detector_pixel_in_lambda_m"] * lam_m / g["pitch_nm"]
    assert abs(px_features - 8) < 0.01
    assert abs(g["fov_pixels_per_side"] * 8 - 200) == 0


def test_experimental_wavelength_list_is_the_small_workload():
    g = _golden()
    w = W.workload("small")
    assert np.allclose(w.lambdas * 1e9, g["experiment_lambdas_nm"], atol=1e-9)
    assert abs(w.pitch - 0.5 * w.lambda_mean) < 1e-18
