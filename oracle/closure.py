"""FP64 oracle of the learned closure (test infrastructure only).

The paper mentions machine-learned reconstruction of turbulent flows from
low-resolution data only in passing (Sec. 6); the closure built here is a
reading of that idea: a three-layer 3-D convolutional net (8 -> 32 -> 32 -> 8
channels, 3x3x3 kernels, circular padding, ReLU after the first two layers)
that maps a coarse state to a correction of it.

Conventions (shared by the CUDA path through the interface, not through code):
  * activations are (C, nz, ny, nx) arrays, x fastest;
  * a weight tensor is W[co, ci, kz, ky, kx]; output cell (z, y, x) takes
    x_in[ci, z + kz - 1, y + ky - 1, x + kx - 1] (indices periodic), i.e. a
    cross-correlation, as in common deep-learning libraries;
  * the loss is the mean squared error over all cells and channels;
  * Adam (Kingma and Ba, 2015) with bias correction.
Plain loops over the 27 taps with NumPy rolls; no blocking or reordering.
"""
import numpy as np

TAPS = [(kz, ky, kx) for kz in range(3) for ky in range(3) for kx in range(3)]


def shifted(x, kz, ky, kx):
    """x[..., z + kz - 1, y + ky - 1, x + kx - 1] with periodic indices."""
    return np.roll(x, shift=(1 - kz, 1 - ky, 1 - kx), axis=(-3, -2, -1))


def conv3d(x, W, b):
    """y[co] = b[co] + sum_{ci, taps} W[co, ci, tap] * shifted(x[ci], tap)."""
    cout = W.shape[0]
    y = np.zeros((cout,) + x.shape[1:])
    for (kz, ky, kx) in TAPS:
        xs = shifted(x, kz, ky, kx)
        y += np.einsum("oi,izyx->ozyx", W[:, :, kz, ky, kx], xs)
    return y + b[:, None, None, None]


def conv3d_input_grad(dy, W):
    """Gradient of sum(dy * conv3d(x, W, b)) with respect to x."""
    cin = W.shape[1]
    dx = np.zeros((cin,) + dy.shape[1:])
    for (kz, ky, kx) in TAPS:
        # x[ci, p + off] contributed to y[co, p]: move dy back by -off
        contrib = np.einsum("oi,ozyx->izyx", W[:, :, kz, ky, kx], dy)
        dx += np.roll(contrib, shift=(kz - 1, ky - 1, kx - 1), axis=(-3, -2, -1))
    return dx


def conv3d_weight_grad(dy, x):
    """Gradients of sum(dy * conv3d(x, W, b)) with respect to W and b."""
    cout, cin = dy.shape[0], x.shape[0]
    dW = np.zeros((cout, cin, 3, 3, 3))
    for (kz, ky, kx) in TAPS:
        xs = shifted(x, kz, ky, kx)
        dW[:, :, kz, ky, kx] = np.einsum("ozyx,izyx->oi", dy, xs)
    db = dy.sum(axis=(1, 2, 3))
    return dW, db


def bf16_round(a):
    """Round binary64 values to bfloat16 (round to nearest even), returned as binary64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class Net:
    """Parameters: list of (W, b) for the three layers."""

    def __init__(self, params):
        self.params = [(np.array(W, dtype=np.float64), np.array(b, dtype=np.float64))
                       for W, b in params]

    @staticmethod
    def init(seed, channels=(8, 32, 32, 8)):
        g = np.random.Generator(np.random.PCG64(seed))
        params = []
        for cin, cout in zip(channels[:-1], channels[1:]):
            bound = 1.0 / np.sqrt(cin * 27)
            W = g.uniform(-bound, bound, size=(cout, cin, 3, 3, 3))
            b = g.uniform(-bound, bound, size=cout)
            params.append((W, b))
        return Net(params)

    # Precision of an evaluation (the `bf16` argument):
    #   None      -- binary64 throughout;
    #   "config"  -- what the configuration fixes: bfloat16 weights (and the
    #                bfloat16 network input, the first layer's operand); every
    #                other value, forward and backward, in binary64;
    #   "kernel"  -- a diagnostic: also bfloat16 wherever the GPU kernels store
    #                an operand in bfloat16 (hidden activations, and in the
    #                backward pass the output gradient and the masked input
    #                gradients), binary64 accumulation.
    # `perturb` (with bf16="config") replaces the rounding at those kernel
    # points by a given function, for the spread estimate below.
    def forward(self, x, bf16=None, perturb=None):
        """Returns (y, activations): the input of every layer."""
        r = bf16_round if bf16 else (lambda a: a)
        rk = perturb or (bf16_round if bf16 == "kernel" else (lambda a: a))
        acts = [r(x)]
        h = acts[0]
        for li, (W, b) in enumerate(self.params):
            z = conv3d(h, r(W), b)
            if li < len(self.params) - 1:
                h = rk(np.maximum(z, 0.0))
                acts.append(h)
            else:
                h = z
        return h, acts

    def loss_and_grads(self, x, target, bf16=None, perturb=None):
        """Mean squared error and its gradients (precision as in forward)."""
        r = bf16_round if bf16 else (lambda a: a)
        rk = perturb or (bf16_round if bf16 == "kernel" else (lambda a: a))
        y, acts = self.forward(x, bf16, perturb)
        n = y.size
        loss = float(np.mean((y - target) ** 2))
        dy = rk(2.0 * (y - target) / n)
        grads = [None] * len(self.params)
        for li in reversed(range(len(self.params))):
            W, b = self.params[li]
            dW, db = conv3d_weight_grad(dy, acts[li])
            grads[li] = (dW, db)
            if li > 0:
                da = conv3d_input_grad(dy, r(W))
                dy = rk(da * (acts[li] > 0))
        return loss, grads

    def rounding_spread(self, x, target=None, samples=16, seed=0):
        """Elementwise standard deviation of the output (target None) or of the
        gradients that bfloat16 rounding at the GPU kernels' rounding points
        produces around the bf16="config" evaluation, under the probabilistic
        model of rounding error (Higham and Mary, SIAM J. Sci. Comput. 41(5),
        2019: each rounding an independent error, here uniform within half a
        bfloat16 unit in the last place of the value, 2^(floor(log2|a|) - 8)),
        estimated from `samples` evaluations with such random errors at those
        points.  Returns sigma of y, or a list of (sigma dW, sigma db) per
        layer."""
        g = np.random.Generator(np.random.PCG64(seed))

        def pert(a):
            a = np.asarray(a, dtype=np.float64)
            half_ulp = np.where(a != 0.0, np.ldexp(1.0, (np.floor(np.log2(np.abs(np.where(
                a != 0.0, a, 1.0)))) - 8).astype(int)), 0.0)
            return a + half_ulp * g.uniform(-1.0, 1.0, size=a.shape)

        runs = []
        for _ in range(samples):
            if target is None:
                runs.append(self.forward(x, "config", pert)[0])
            else:
                runs.append(self.loss_and_grads(x, target, "config", pert)[1])
        if target is None:
            return np.std(np.stack(runs), axis=0, ddof=1)
        return [tuple(np.std(np.stack([rr[li][a] for rr in runs]), axis=0, ddof=1)
                      for a in range(2)) for li in range(len(self.params))]

    def flat(self):
        """Parameters as one vector: W1, b1, W2, b2, W3, b3 (row-major)."""
        return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in self.params])

    @staticmethod
    def unflat(v, channels=(8, 32, 32, 8)):
        params, o = [], 0
        for cin, cout in zip(channels[:-1], channels[1:]):
            nW = cout * cin * 27
            W = np.array(v[o:o + nW], dtype=np.float64).reshape(cout, cin, 3, 3, 3)
            o += nW
            b = np.array(v[o:o + cout], dtype=np.float64)
            o += cout
            params.append((W, b))
        return Net(params)


class Adam:
    """Adam with bias correction: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, shapes, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = [np.zeros(s) for s in shapes]
        self.v = [np.zeros(s) for s in shapes]
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            out.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out


def energy_spectrum(v, n=None):
    """Shell-summed spectrum E(k) = sum_{|kappa| in [k-1/2, k+1/2)} |v_hat(kappa)|^2 / 2
    of a vector field v (3, nz, ny, nx), FFT normalised by 1/N (a diagnostic)."""
    shape = v.shape[1:]
    N = np.prod(shape)
    vh = [np.fft.fftn(v[a]) / N for a in range(3)]
    e = 0.5 * sum(np.abs(h) ** 2 for h in vh)
    ks = np.meshgrid(*[np.fft.fftfreq(m, 1.0 / m) for m in shape], indexing="ij")
    kk = np.sqrt(sum(k ** 2 for k in ks))
    kmax = int(np.max(kk)) + 1 if n is None else n
    shells = np.floor(kk + 0.5).astype(int)
    return np.bincount(shells.ravel(), weights=e.ravel(), minlength=kmax + 1)[:kmax + 1]
