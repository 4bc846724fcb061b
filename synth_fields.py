"""Seeded synthetic scalar fields: stand-ins for the SDRBench fields of Table 1.

This module only makes inputs.  It holds none of the compression method's
arithmetic (no ranges, no tolerance schedules, no coding) and it is the one
module that both the CPU oracle's tests and the GPU path's tests and bench
import.  Every generator is seeded with numpy's PCG64.

Arrays are C-ordered with shape (nz, ny, nx) for 3D (x fastest), (ny, nx) for
2D and (nx,) for 1D.

Recipes (the shapes and precisions mirror Table 1's Miranda 384x384x256 f64
and Nyx 512^3 f32; the data themselves are not available):
  * gaussians: a sum of random anisotropic Gaussians, centres uniform in the
    box, per-axis widths uniform in [2, 16] cells, amplitudes uniform in
    (-1, 1), plus N(0, noise^2) white noise.
  * powerlaw: a random-phase Gaussian field with power spectrum k^-5/3:
    Fourier amplitude |k|^-5/6, phases uniform in [0, 2pi), k = 0 removed,
    real inverse FFT, scaled to unit variance.
  * fronts: powerlaw plus sharp tanh interfaces sum_j a_j tanh((n_j.r - c_j)/w)
    with w = 1 cell, enough of them that |grad| is large on about 1% of cells.
"""
import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussians(shape, n_gauss: int = 32, seed: int = 1, dtype=np.float64, noise: float = 1e-3, device=None):
    """Sum of n_gauss random anisotropic Gaussians plus white noise.

    device=None builds it with numpy and returns a numpy array; device="cuda"
    builds it with torch there (same Gaussians; the noise comes from torch's
    generator seeded with `seed`) and returns a torch tensor."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    if device is not None:
        return _gaussians_torch(shape, n_gauss, seed, rng, dtype, noise, device)
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    out = np.zeros(shape, dtype=np.float64)
    for _ in range(n_gauss):
        centre = [rng.uniform(0, s) for s in shape]
        sigma = [rng.uniform(2.0, 16.0) for _ in shape]
        amp = rng.uniform(-1.0, 1.0)
        g = None
        for a in range(nd):
            prof = np.exp(-0.5 * ((axes[a] - centre[a]) / sigma[a]) ** 2)
            view = [1] * nd
            view[a] = shape[a]
            prof = prof.reshape(view)
            g = prof if g is None else g * prof
        out += amp * g
    if noise:
        out += rng.normal(0.0, noise, size=shape)
    return out.astype(dtype)


def _gaussians_torch(shape, n_gauss, seed, rng, dtype, noise, device):
    import torch

    nd = len(shape)
    axes = [torch.arange(s, device=device, dtype=torch.float64) for s in shape]
    out = torch.zeros(shape, device=device, dtype=torch.float64)
    for _ in range(n_gauss):
        centre = [rng.uniform(0, s) for s in shape]
        sigma = [rng.uniform(2.0, 16.0) for _ in shape]
        amp = rng.uniform(-1.0, 1.0)
        g = None
        for a in range(nd):
            prof = torch.exp(-0.5 * ((axes[a] - centre[a]) / sigma[a]) ** 2)
            view = [1] * nd
            view[a] = shape[a]
            prof = prof.reshape(view)
            g = prof if g is None else g * prof
        out += amp * g
    if noise:
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        out += noise * torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
    return out.to(torch.float32 if np.dtype(dtype) == np.float32 else torch.float64)


def _powerlaw_numpy(shape, rng):
    freqs = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*freqs, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    k2[(0,) * len(shape)] = 1.0
    amp = k2 ** (-5.0 / 12.0)  # |k|^(-5/6)
    amp[(0,) * len(shape)] = 0.0
    phase = rng.uniform(0.0, 2.0 * np.pi, size=amp.shape)
    spec = amp * np.exp(1j * phase)
    del phase, amp, k2
    f = np.fft.irfftn(spec, s=shape, axes=tuple(range(len(shape))))
    f -= f.mean()
    f /= f.std()
    return f


def _powerlaw_torch(shape, rng, device):
    import torch

    dev = torch.device(device)
    freqs = [torch.fft.fftfreq(s, device=dev, dtype=torch.float64) for s in shape[:-1]]
    freqs.append(torch.fft.rfftfreq(shape[-1], device=dev, dtype=torch.float64))
    half = tuple(shape[:-1]) + (shape[-1] // 2 + 1,)
    k2 = torch.zeros(half, device=dev, dtype=torch.float64)
    for a, fr in enumerate(freqs):
        view = [1] * len(shape)
        view[a] = fr.numel()
        k2 += fr.reshape(view) ** 2
    k2.view(-1)[0] = 1.0
    amp = k2.pow_(-5.0 / 12.0)
    amp.view(-1)[0] = 0.0
    # phases drawn on the host from the seeded generator, one z-slab at a time
    spec = torch.empty(half, device=dev, dtype=torch.complex128)
    for z in range(half[0]):
        ph = torch.from_numpy(rng.uniform(0.0, 2.0 * np.pi, size=half[1:])).to(dev)
        spec[z] = torch.polar(amp[z], ph)
    del amp, k2
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    f -= f.mean()
    f /= f.std()
    return f


def powerlaw(shape, seed: int = 2, dtype=np.float32, device=None):
    """Random-phase Gaussian field with P(k) ~ k^-5/3 and unit variance.

    device=None builds it with numpy on the host and returns a numpy array;
    device="cuda" builds it with torch.fft there and returns a torch tensor
    (for fields too large to build quickly on the host)."""
    rng = _rng(seed)
    shape = tuple(int(s) for s in shape)
    if device is None:
        return _powerlaw_numpy(shape, rng).astype(dtype)
    import torch

    f = _powerlaw_torch(shape, rng, device)
    return f.to(torch.float32 if np.dtype(dtype) == np.float32 else torch.float64)


def fronts(shape, seed: int = 5, dtype=np.float64, n_fronts: int = 24, device=None):
    """powerlaw plus sharp tanh interfaces (planes and spheres), width 1 cell."""
    rng = _rng(seed + 1000)
    shape = tuple(int(s) for s in shape)
    base = powerlaw(shape, seed=seed, dtype=np.float64, device=device)
    specs = []
    for j in range(n_fronts):
        amp = rng.uniform(-2.0, 2.0)
        if j % 2 == 0:  # plane through a random point with a random normal
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            c = float(np.dot(nrm, [rng.uniform(0, s) for s in shape[::-1]]))
            specs.append(("plane", amp, nrm, c))
        else:  # sphere
            ctr = np.array([rng.uniform(0, s) for s in shape[::-1]])
            rad = rng.uniform(0.05, 0.3) * min(shape)
            specs.append(("sphere", amp, ctr, rad))
    if device is None:
        zz, yy, xx = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij", sparse=True)
        for kind, amp, a, b in specs:
            if kind == "plane":
                base += amp * np.tanh(a[0] * xx + a[1] * yy + a[2] * zz - b)
            else:
                r = np.sqrt((xx - a[0]) ** 2 + (yy - a[1]) ** 2 + (zz - a[2]) ** 2)
                base += amp * np.tanh(r - b)
        return base.astype(dtype)
    import torch

    dev = base.device
    xs = [torch.arange(s, device=dev, dtype=torch.float64) for s in shape]
    for z in range(shape[0]):  # slab by slab to bound the temporaries
        yy = xs[1].view(-1, 1)
        xx = xs[2].view(1, -1)
        zz = float(z)
        sl = base[z]
        for kind, amp, a, b in specs:
            if kind == "plane":
                sl += amp * torch.tanh(a[0] * xx + a[1] * yy + a[2] * zz - b)
            else:
                r = torch.sqrt((xx - a[0]) ** 2 + (yy - a[1]) ** 2 + (zz - a[2]) ** 2)
                sl += amp * torch.tanh(r - b)
    return base.to(torch.float32 if np.dtype(dtype) == np.float32 else torch.float64)


def batched_shapes(count: int = 64, seed: int = 3):
    """Shapes of the uneven batch: half 2D with extents in [256, 4096], half 3D
    between 32^3 and 384x384x256; extents are not forced to multiples of 4."""
    rng = _rng(seed)
    shapes = []
    for i in range(count):
        if i % 2 == 0:
            shapes.append((int(rng.integers(256, 4097)), int(rng.integers(256, 4097))))
        else:
            shapes.append((int(rng.integers(32, 257)), int(rng.integers(32, 385)), int(rng.integers(32, 385))))
    return shapes
