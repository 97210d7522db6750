"""The largest transforms a plan allows (p^m <= 2^31): p = 2, m = 31,
p = 3, m = 19 and p = 31, m = 6, on characters of the digit group, whose transforms are known
exactly.  For p = 2 the input f_n = (-1)^(n . h*) keeps every intermediate of
the butterflies at 0 or +-2^k, so the forward result is the unit vector at h*
bit for bit, and the inverse gives f back bit for bit (Sec. 2.2: the Walsh
functions are the characters, and the transform is the Kronecker power of the
p-point DFT)."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu

CHUNK = 1 << 27


def _parity(x):
    for sh in (32, 16, 8, 4, 2, 1):
        x = x ^ (x >> sh)
    return x & 1


def test_p2_m31_walsh_function_exact(dwt, dev):
    p, m = 2, 31
    N = 1 << m
    free, _ = torch.cuda.mem_get_info()
    if free < 3 * 4 * N:
        pytest.skip("needs about 26 GB of device memory")
    h = int(S.integers(S.stream_seed(70, S.P_SAMPLE, 0), 1, 1, N - 1)[0])
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=3), dwt.DWT_PLAN_TRANSFORM_ONLY)
    f = torch.empty(N, dtype=torch.float32, device=dev)
    for a in range(0, N, CHUNK):
        n = torch.arange(a, min(N, a + CHUNK), dtype=torch.int64, device=dev)
        f[a:a + n.numel()] = (1 - 2 * _parity(n & h)).to(torch.float32)
        del n
    g = torch.empty_like(f)
    dwt.dwt_forward(plan, f, g, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
    assert float(g[h]) == 1.0
    assert int(torch.count_nonzero(g)) == 1
    dwt.dwt_inverse(plan, g, g, 1, N, N, dwt.DWT_F32, dwt.DWT_F32)
    assert bool(torch.equal(g, f))


@pytest.mark.parametrize("p,m", [(3, 19), (31, 6)])
def test_p_odd_max_character(dwt, dev, p, m):
    N = p ** m
    ld = (N + 3) // 4 * 4
    free, _ = torch.cuda.mem_get_info()
    if free < 3 * 8 * ld:
        pytest.skip("needs about 30 GB of device memory")
    hd = S.integers(S.stream_seed(71, S.P_SAMPLE, p), m, 0, p - 1)      # digits of h*
    hd[0] = 1
    h = int(sum(int(d) * p ** i for i, d in enumerate(hd)))
    plan = dwt.dwt_plan_create(p, m, 1, S.small_net(p, m, 1, index=4), dwt.DWT_PLAN_TRANSFORM_ONLY)
    # f_n = omega^(n . h*), omega = exp(2 pi i / p): its forward transform (omega^(-n . h)) is the unit vector at h*
    f = torch.zeros(2 * ld, dtype=torch.float32, device=dev)
    fc = f.view(torch.complex64)
    w = torch.exp(2j * np.pi * torch.arange(p, dtype=torch.float64, device=dev) / p).to(torch.complex64)
    for a in range(0, N, CHUNK):
        n = torch.arange(a, min(N, a + CHUNK), dtype=torch.int64, device=dev)
        e = torch.zeros_like(n)
        v = n.clone()
        for i in range(m):
            e += (v % p) * int(hd[i])
            v //= p
        fc[a:a + n.numel()] = w[e % p]
        del n, e, v
    g = torch.empty_like(f)
    dwt.dwt_forward(plan, f, g, 1, ld, ld, dwt.DWT_C64, dwt.DWT_C64)
    gc = g.view(torch.complex64)[:N]
    assert abs(complex(gc[h]) - 1.0) < 1e-5
    gc[h] = 0
    assert float(gc.abs().max()) < 1e-5
