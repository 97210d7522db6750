"""One transform split across G = p^g processes, with one all-to-all exchange.

The transform of Sec. 2.2 is the Kronecker product of one p-point DFT per
index digit (the nested-sum form of eq. fdwt), and the stages of different
digits commute (Algorithm 1 runs them in any order).  Cutting the digits at
m - g gives a transform of N = p^m points on G = p^g processes:

 * process r holds the N / G consecutive samples whose top g digits equal r,
   n = n_lo + p^(m-g) r;
 * it runs the stages of its m - g low digits on its block (a transform of
   p^(m-g) points; forward factor p^-(m-g));
 * one all-to-all: piece r' (p^(m-2g) consecutive values) of every block goes
   to process r', which stores the piece from process r at offset r p^(m-2g);
 * it runs the stages of digits m-2g .. m-g-1 of the received block, which are
   the sender index r, i.e. the top g digits of n (forward factor p^-g).

Afterwards process r' holds f~(H) for the H whose low m - g digits lie in
[r' p^(m-2g), (r'+1) p^(m-2g)): H = (r' p^(m-2g) + j) + p^(m-g) h at offset
h p^(m-2g) + j.  The inverse (Algorithm 2) runs the same steps backwards; the
exchange pattern is its own inverse.  Needs m >= 2 g.

The local stages run in the library's kernels (dwt_forward_digits /
dwt_inverse_digits on a plan of p^(m-g) points); the exchange is a collective
of the caller's process group (torch.distributed.all_to_all_single), or any
function with the same contract.  This module only arranges the calls.
"""
import paper_0808_0487_gb300 as _dwt


def block_of(rank, p, m, g):
    """The sample indices n held by process ``rank``: [rank p^(m-g), (rank+1) p^(m-g))."""
    L = p ** (m - g)
    return rank * L, (rank + 1) * L


def coefficient_index(rank, p, m, g):
    """Coefficient label H of every offset of process ``rank``'s result, as a list."""
    chunk = p ** (m - 2 * g)
    L = p ** (m - g)
    G = p ** g
    return [rank * chunk + j + L * h for h in range(G) for j in range(chunk)]


class LibraryStages:
    """Digit stages of a local block of p^(m-g) points with the library's kernels.
    Blocks are torch tensors on the device: float32 for p = 2, complex64 for
    p > 2 (the forward of the low digits also takes real float32 input)."""

    def __init__(self, p, m_local, stream=None):
        import numpy as np
        self.p = p
        self.m = m_local
        self.N = p ** m_local
        self.stream = stream
        C = np.zeros((1, m_local, m_local), dtype=np.uint8)
        for i in range(m_local):
            C[0, i, m_local - 1 - i] = 1
        self.plan = _dwt.dwt_plan_create(p, m_local, 1, C, _dwt.DWT_PLAN_TRANSFORM_ONLY)

    def __call__(self, inp, out, d0, nd, sgn):
        import torch
        p = self.p
        if p == 2:
            ti = to = _dwt.DWT_F32
        else:
            ti = _dwt.DWT_F32 if inp.dtype == torch.float32 else _dwt.DWT_C64
            to = _dwt.DWT_C64
        call = _dwt.dwt_forward_digits if sgn < 0 else _dwt.dwt_inverse_digits
        call(self.plan, inp, out, 1, self.N, self.N, ti, to, d0, nd, stream=self.stream)


def torch_exchange(group=None):
    """The all-to-all of the process group: equal pieces, piece i to rank i."""
    import torch
    import torch.distributed as dist

    def ex(send, recv):
        s = torch.view_as_real(send).reshape(-1) if send.is_complex() else send
        r = torch.view_as_real(recv).reshape(-1) if recv.is_complex() else recv
        dist.all_to_all_single(r, s, group=group)

    return ex


class ShardedTransform:
    """The forward and inverse transform of N = p^m points on G = p^g processes."""

    def __init__(self, p, m, g, stages, exchange):
        if g < 0 or m < 2 * g:
            raise ValueError("a cut at digit m - g needs m >= 2 g")
        self.p, self.m, self.g = p, m, g
        self.G = p ** g
        self.L = p ** (m - g)
        self.stages = stages
        self.exchange = exchange

    # the steps on one process, in order (forward: low, exchange, top; inverse:
    # top_inverse, exchange, low_inverse)
    def low(self, x, work):
        self.stages(x, work, 0, self.m - self.g, -1)

    def top(self, buf):
        if self.g:
            self.stages(buf, buf, self.m - 2 * self.g, self.g, -1)

    def top_inverse(self, c, work):
        if self.g:
            self.stages(c, work, self.m - 2 * self.g, self.g, +1)

    def low_inverse(self, buf):
        self.stages(buf, buf, 0, self.m - self.g, +1)

    def forward(self, x, work, out):
        """x: this process's block (n order); work, out: blocks of the result type.
        out receives this process's coefficients (see the module docstring)."""
        if not self.g:
            self.stages(x, out, 0, self.m, -1)
            return out
        self.low(x, work)
        self.exchange(work, out)                      # piece r' -> process r'
        self.top(out)                                 # the sender digits = top digits of n
        return out

    def inverse(self, c, work, out):
        """c: this process's coefficients (layout of forward); out: its block (n order)."""
        if not self.g:
            self.stages(c, out, 0, self.m, +1)
            return out
        self.top_inverse(c, work)
        self.exchange(work, out)
        self.low_inverse(out)
        return out
