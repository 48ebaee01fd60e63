"""GPU checks of the integer issue probes (spvar_measure_issue_rate), the
measured ceilings of the sweep kernels' rooflines: every form runs and
reports a rate below the SM count x 128 lanes x the maximum SM clock, and
a Philox4x32-10 block costs about twenty of the wide-multiply probe's
operations (each of them one wide multiply and one three-input xor, as in a
Philox round)."""
import pytest

pytestmark = pytest.mark.gpu


def test_issue_probes_are_bounded_and_consistent(cuda_lib):
    import torch
    spvar = cuda_lib
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 128 * 2.2e9
    rates = {}
    for form in range(6):
        r, ms = spvar.measure_issue_rate(form, 256)
        assert r > 0 and ms > 0, form
        rates[form] = r
    for form in range(5):
        assert rates[form] < 1.05 * bound, (form, rates[form], bound)
    # both pipes together issue at least as fast as either alone
    assert rates[3] > 0.9 * max(rates[0], rates[2])
    ratio = rates[4] / (20 * rates[5])
    assert 0.6 < ratio < 1.6, ratio
    with pytest.raises(spvar.SpvarError):
        spvar.measure_issue_rate(6, 10)
