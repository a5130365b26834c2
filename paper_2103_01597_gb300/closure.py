"""Learned closure: training pairs from the solver, training, rollout.

This module sequences calls into libac.so (restriction, solver steps, closure
forward/backward/Adam/apply kernels) and holds torch-owned device buffers.
Every step of the solver and of the network runs in the library's CUDA
kernels.  Two pieces of training-data preparation, outside any timed step, are
torch tensor operations: the target defect (restricted fine state minus the
coarse step, one subtraction on the device) and the per-channel rms of the
training set used as the network's input and output scales (channel_rms).

Data (a reading; the paper only mentions learned reconstruction, Sec. 6): a
fine binary64 run on a grid 2x finer per axis, restricted by full weighting.
For each pair, input = R(f_fine(t)) and target = R(f_fine(t + 2 dt)) minus
one binary32 coarse step of 2 dt from R(f_fine(t)).  The forcing is drawn
once per coarse step and applied to the fine run's two steps and the coarse
step alike, so the target holds no unpredictable forcing.
"""
import math

import numpy as np

from . import ac


def init_params(seed):
    """Seeded uniform initialisation, bound 1/sqrt(fan_in) per layer (host)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for cin, cout in ((8, 32), (32, 32), (32, 8)):
        bound = 1.0 / math.sqrt(cin * 27)
        out.append(g.uniform(-bound, bound, size=cout * cin * 27))
        out.append(g.uniform(-bound, bound, size=cout))
    return np.concatenate(out).astype(np.float32)


def _rows(t):
    return [t[q].data_ptr() for q in range(8)]


def current_state(sim):
    """torch view (8, elems) of a Simulation's current state buffer."""
    ptrs, _, _, _ = ac.ac_get_state(sim.h)
    for b in range(2):
        if sim.state[b, 0].data_ptr() == ptrs[0]:
            return sim.state[b, :, :sim.elems]
    raise RuntimeError("current state is not one of the bound buffers")


class Closure:
    def __init__(self, n, seed=0, params=None, stream=None, conv_path=ac.AC_CONV_TCGEN05):
        import torch
        self.n = tuple(n)
        self.cells = n[0] * n[1] * n[2]
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.c = ac.ac_closure_init(n, stream)
        ac.ac_closure_set_conv_path(self.c, conv_path)
        ac.ac_closure_set_params(self.c, init_params(seed) if params is None else params)
        self.out = torch.zeros((8, self.cells), dtype=torch.float32, device="cuda")

    def set_scales(self, in_scale, out_scale):
        ac.ac_closure_set_scales(self.c, in_scale, out_scale)

    def correction(self, x):
        ac.ac_closure_forward(self.c, _rows(x), _rows(self.out))
        return self.out

    def train_step(self, x, target, lr):
        loss = ac.ac_closure_backward(self.c, _rows(x), _rows(target))
        ac.ac_closure_adam_step(self.c, lr)
        return loss

    def loss(self, x, target):
        return ac.ac_closure_backward(self.c, _rows(x), _rows(target))

    def apply(self, sim, limit):
        return ac.ac_closure_apply(self.c, sim.h, limit)

    def status(self):
        """Raise AcError if a bounded wait of the tensor-core kernels ran out."""
        ac.ac_closure_status(self.c)

    def close(self):
        if self.c is not None:
            ac.ac_closure_quit(self.c)
            self.c = None


def make_pairs(f0, n_fine, npairs, dt_fine, seed=0, force_amp=0.0, warm_steps=0,
               nu=5e-3, eta=5e-3):
    """Training pairs (input, target) as torch (8, cells) binary32 tensors on the
    coarse grid, from a fine binary64 run started at f0 (host array)."""
    import torch
    n_c = tuple(v // 2 for v in n_fine)
    cells = n_c[0] * n_c[1] * n_c[2]
    fine = ac.Simulation(n_fine, precision=ac.AC_FP64, nu=nu, eta=eta, force_amp=force_amp,
                         seed=seed)
    coarse = ac.Simulation(n_c, precision=ac.AC_FP32, nu=nu, eta=eta, force_amp=force_amp,
                           seed=seed)
    fine.load(f0)
    for _ in range(warm_steps):
        fine.step(dt_fine)
    pairs = []
    nxt = torch.empty((8, cells), dtype=torch.float32, device="cuda")
    for p in range(npairs):
        if force_amp:
            frc = ac.ac_forcing_draw(seed, 1000 + p)
            ac.ac_set_forcing(fine.h, *frc)
            ac.ac_set_forcing(coarse.h, *frc)
        x = torch.empty((8, cells), dtype=torch.float32, device="cuda")
        fptrs, _, _, _ = ac.ac_get_state(fine.h)
        ac.ac_restrict(fptrs, ac.AC_FP64, n_fine, _rows(x))
        fine.step(dt_fine)
        fine.step(dt_fine)
        ac.ac_last_cfl(fine.h)  # raises if the fine run stopped being finite
        fptrs, _, _, _ = ac.ac_get_state(fine.h)
        ac.ac_restrict(fptrs, ac.AC_FP64, n_fine, _rows(nxt))
        current_state(coarse).copy_(x)
        coarse.step(2 * dt_fine)
        target = nxt - current_state(coarse)
        pairs.append((x, target))
    torch.cuda.synchronize()
    fine.close()
    coarse.close()
    return pairs


def channel_rms(tensors):
    """Per-channel rms over a list of (8, cells) tensors (host floats; torch
    reductions on the device, data preparation only)."""
    acc = np.zeros(8)
    count = 0
    for t in tensors:
        acc += (t.double() ** 2).sum(dim=1).cpu().numpy()
        count += t.shape[1]
    r = np.sqrt(acc / count)
    return np.where(r > 0, r, 1.0).astype(np.float32)
