"""dwt_interpolate_host: host-resident samples and results with the copies
overlapped with the transforms.  The device path (dwt_interpolate) is itself
checked against the oracle elsewhere; here the host path must reproduce it bit
for bit, over several chunks (slot reuse), padded rows, complex output and
pageable buffers."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _device_run(dwt, dev, plan, f_host, batch, ld, f_t, c_dtype, s):
    f = torch.from_numpy(f_host).to(dev)
    c = torch.zeros((batch, ld), dtype=c_dtype, device=dev)
    var = torch.empty((batch, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((batch, 2), dtype=torch.int32, device=dev)
    dwt.dwt_interpolate(plan, f, c, None, batch, ld, f_t, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    torch.cuda.synchronize()
    return c.cpu().numpy(), var.cpu().numpy(), dim.cpu().numpy()


def _host_run(dwt, plan, f_host, batch, ld, f_t, c_np_dtype, s, pinned):
    if pinned:
        f_t_ = torch.from_numpy(f_host).pin_memory()
        c_t = torch.zeros((batch, ld), dtype=torch.float32 if c_np_dtype == np.float32 else torch.complex64).pin_memory()
        var_t = torch.empty((batch, 2, s + 1), dtype=torch.float64).pin_memory()
        dim_t = torch.empty((batch, 2), dtype=torch.int32).pin_memory()
        dwt.dwt_interpolate_host(plan, f_t_, c_t, batch, ld, f_t, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var_t, dim=dim_t)
        torch.cuda.synchronize()
        return c_t.numpy(), var_t.numpy(), dim_t.numpy()
    c = np.zeros((batch, ld), dtype=c_np_dtype)
    var = np.empty((batch, 2, s + 1), dtype=np.float64)
    dim = np.empty((batch, 2), dtype=np.int32)
    dwt.dwt_interpolate_host(plan, f_host, c, batch, ld, f_t, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=var, dim=dim)
    torch.cuda.synchronize()
    return c, var, dim


def _product_samples(dwt, dev, plan, coef, batch, ld):
    f = torch.zeros((batch, ld), dtype=torch.float32, device=dev)
    dwt.dwt_eval_product(plan, torch.tensor(coef, dtype=torch.float64, device=dev), f, batch, ld, dwt.DWT_F32)
    torch.cuda.synchronize()
    return np.ascontiguousarray(f.cpu().numpy())


@pytest.mark.parametrize("m,s,batch,ld_pad,pinned", [(24, 32, 5, 0, True), (20, 16, 37, 0, True),
                                                     (16, 8, 3, 12, False), (13, 5, 4, 4, True)])
def test_host_matches_device_p2(dwt, dev, m, s, batch, ld_pad, pinned):
    p = 2
    N = 2 ** m
    ld = N + ld_pad
    C = S.small_net(p, m, s, index=40 + m)
    plan = dwt.dwt_plan_create(p, m, s, C)
    coef = S.uniform(S.stream_seed(40, S.P_COEFFS, m), batch * s).reshape(batch, s)
    f_host = _product_samples(dwt, dev, plan, coef, batch, ld)
    c_ref, var_ref, dim_ref = _device_run(dwt, dev, plan, f_host, batch, ld, dwt.DWT_F32, torch.float32, s)
    c, var, dim = _host_run(dwt, plan, f_host, batch, ld, dwt.DWT_F32, np.float32, s, pinned)
    assert np.array_equal(c[:, :N].view(np.uint32), c_ref[:, :N].view(np.uint32))
    assert np.array_equal(var.view(np.uint64), var_ref.view(np.uint64))
    assert np.array_equal(dim, dim_ref)
    # a second call on the same plan with a larger batch reuses the slots
    f2 = np.concatenate([f_host, f_host[::-1]])
    c2, var2, dim2 = _host_run(dwt, plan, f2, 2 * batch, ld, dwt.DWT_F32, np.float32, s, pinned)
    assert np.array_equal(c2[:batch, :N].view(np.uint32), c_ref[:, :N].view(np.uint32))
    assert np.array_equal(c2[batch:, :N].view(np.uint32), c_ref[::-1, :N].view(np.uint32))
    assert np.array_equal(dim2[batch:], dim_ref[::-1])


def test_host_matches_device_p3_complex(dwt, dev):
    p, m, s, batch = 3, 9, 6, 4
    N = p ** m
    ld = N + 5
    C = S.small_net(p, m, s, index=41)
    plan = dwt.dwt_plan_create(p, m, s, C)
    coef = S.uniform(S.stream_seed(41, S.P_COEFFS), batch * s).reshape(batch, s)
    f_host = _product_samples(dwt, dev, plan, coef, batch, ld)
    c_ref, var_ref, dim_ref = _device_run(dwt, dev, plan, f_host, batch, ld, dwt.DWT_F32, torch.complex64, s)
    c, var, dim = _host_run(dwt, plan, f_host, batch, ld, dwt.DWT_F32, np.complex64, s, True)
    assert np.array_equal(c[:, :N].view(np.uint64), c_ref[:, :N].view(np.uint64))
    assert np.array_equal(var.view(np.uint64), var_ref.view(np.uint64))
    assert np.array_equal(dim, dim_ref)


def test_host_bad_arguments(dwt, dev):
    C = S.small_net(2, 12, 3, index=42)
    plan = dwt.dwt_plan_create(2, 12, 3, C)
    f = np.zeros((1, 4096), dtype=np.float32)
    with pytest.raises(dwt.DwtError):
        dwt.dwt_interpolate_host(plan, f, None, 1, 4096, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER)
    with pytest.raises(dwt.DwtError):
        dwt.dwt_interpolate_host(plan, f, f, 1, 4095, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER)
