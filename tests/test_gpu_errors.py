"""Failure handling on the GPU without any fault: bounded wavefront waits that
run out (a row counter nothing sets), non-physical inputs and bad arguments
all come back as status codes, and the problem stays usable afterwards."""
import numpy as np
import pytest

from _cases import build_case, config, rel_err, run_gpu

pytestmark = pytest.mark.gpu


def test_wait_timeout_reports_status_and_recovers(gpu_lib):
    cfg = config(2, 32, 24, 4, 2, 4)
    case = build_case(gpu_lib, cfg, 32, seed=1, strip_width=8, prefetch_rows=2)
    I_ok, m_ok, _, _ = run_gpu(case)
    prob = case.prob
    prob.debug_wait_limit_ns(50_000_000)  # 50 ms
    prob.debug_skip_publish(True)
    with pytest.raises(gpu_lib.SMError) as ei:
        run_gpu(case)
    assert ei.value.code == 6  # SM_ERR_TIMEOUT
    prob.debug_skip_publish(False)
    prob.debug_wait_limit_ns(2_000_000_000)
    I2, m2, _, _ = run_gpu(case)
    assert np.array_equal(I2, I_ok)
    assert rel_err(m2[..., 0], m_ok[..., 0], 1e-6) < 1e-6


def test_nonphysical_temperature_is_reported(gpu_lib):
    import torch
    cfg = config(2, 8, 8, 2, 1, 2)
    case = build_case(gpu_lib, cfg, 64, seed=2)
    T = case.T.copy()
    T[3, 1] = 0.0
    prob = case.prob
    prob.sweep(torch.from_numpy(T).cuda(), torch.from_numpy(case.sigma).cuda(), None,
               prob.empty_intensity(), prob.new_moments(), None)
    with pytest.raises(gpu_lib.SMError) as ei:
        prob.synchronize()
    assert ei.value.code == 5  # SM_ERR_NONPHYSICAL
    prob.synchronize()  # status was cleared


def test_bad_arguments(gpu_lib):
    import torch
    cfg = config(2, 8, 8, 2, 1, 2)
    case = build_case(gpu_lib, cfg, 32, seed=3)
    prob = case.prob
    I = prob.empty_intensity()
    Td = torch.from_numpy(case.T).cuda()
    Sd = torch.from_numpy(case.sigma).cuda()
    with pytest.raises(gpu_lib.SMError) as ei:
        prob.sweep(Td, Sd, I, I, None, None)  # aliasing
    assert ei.value.code == 1
    with pytest.raises(gpu_lib.SMError):
        prob.set_tiling(100, 2)
    with pytest.raises(gpu_lib.SMError):
        gpu_lib.Problem.from_config(config(2, 0, 4, 2, 1, 1), 32)
