"""The roofline denominators: fp_measure_rates runs and returns plausible
sustained rates (positive, ordered as the hardware's unit counts imply)."""
import pytest

import paper_1307_5655_gb300 as fpl


@pytest.mark.gpu
def test_measure_rates():
    r = fpl.fp_measure_rates()
    assert set(r) == set(fpl.RATE_NAMES)
    assert all(v > 0 for v in r.values()), r
    # FP32 lanes outnumber FP64 ones many times over; a compensated
    # multiply-add is about a dozen FP32 operations, fewer in Horner's form
    assert r["ffma"] > 10 * r["dfma"]
    assert r["f32c_mad"] < r["ffma"] / 6
    assert r["f32c_mad"] < r["f32c_horner"] < r["ffma"] / 6
    # integer multiply-adds: GB300's FP64 rate is far below its integer one,
    # and a 64-bit product mod p takes several 32 x 32 partial products
    assert r["imad"] > 4 * r["dfma"]
    assert r["imad_wide"] > r["modp_muladd"]
