"""Seeded synthetic CP problems shaped like the paper's difficult cases.

This module only draws random inputs: factor matrices (Gaussian, collinear,
scaled), the tensor built from them, additive noise and initial factors.  It
holds none of the damped Gauss-Newton arithmetic, imports neither the CUDA
binding nor the oracle, and is shared by both sides of every parity test.

Conventions: a tensor is a numpy array of shape ``(I_1, ..., I_N)`` whose
``vec`` is column-major (first index fastest), so it is passed to the C ABI
as ``np.asfortranarray(Y)`` / ``Y.ravel(order="F")``.  Factors are float64
``I_n x R`` arrays.

Recipes (paper Sec. 6 and the benchmark configurations):
  * ``paper_collinear``: Eq. (modify_1), a_r = u_1 + nu * u_r with U orthonormal;
    optional magnitudes lambda_1 = 1, lambda_r = (1 + nu^2)^(N/2) (Sec. 6).
  * ``collinear_columns``: a_r = sqrt(c) b + sqrt(1 - c) z_r with b, z_r iid
    N(0, I): expected cosine c between columns.
  * column norms scaled log-uniformly over [lo, hi].
  * noise at a given SNR: sigma = 10^(-SNR/20) ||Y||_F / sqrt(prod I_n)
    (Sec. 6, SNR = 10 log10(||Y||^2 / (sigma^2 prod I_n))).
"""
from __future__ import annotations

import dataclasses
import math
import string
from typing import List, Optional, Sequence

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator; every input of every test and benchmark is seeded."""
    return np.random.default_rng(seed)


def gaussian_factors(rng, dims: Sequence[int], R: int) -> List[np.ndarray]:
    return [rng.standard_normal((I, R)) for I in dims]


def collinear_columns(rng, I: int, R: int, c: float) -> np.ndarray:
    """Columns a_r = sqrt(c) b + sqrt(1-c) z_r; E[cos(a_q, a_r)] ~ c."""
    b = rng.standard_normal((I, 1))
    z = rng.standard_normal((I, R))
    return math.sqrt(c) * b + math.sqrt(1.0 - c) * z


def paper_collinear(rng, I: int, R: int, nu: float) -> np.ndarray:
    """Eq. (modify_1): A = U Q with U (I x R) orthonormal, a_1 = u_1,
    a_r = u_1 + nu u_r for r > 1 (requires I >= R)."""
    U, _ = np.linalg.qr(rng.standard_normal((I, R)))
    A = U.copy()
    A[:, 1:] = U[:, :1] + nu * U[:, 1:]
    return A


def paper_magnitudes(R: int, N: int, nu: float) -> np.ndarray:
    """Sec. 6 magnitude variant: lambda_1 = 1, lambda_r = (1 + nu^2)^(N/2)."""
    lam = np.full(R, (1.0 + nu * nu) ** (N / 2.0))
    lam[0] = 1.0
    return lam


def log_uniform_column_scale(rng, A: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Scale each column to norm 10^U[log10 lo, log10 hi] (direction kept)."""
    R = A.shape[1]
    target = 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=R)
    norms = np.linalg.norm(A, axis=0)
    norms[norms == 0] = 1.0
    return A * (target / norms)[None, :]


def tensor_from_factors(factors: Sequence[np.ndarray],
                        weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Dense sum of R outer products, built with einsum (input synthesis only)."""
    N = len(factors)
    letters = string.ascii_lowercase[:N]
    R = factors[0].shape[1]
    w = np.ones(R) if weights is None else np.asarray(weights, dtype=np.float64)
    spec = ",".join(f"{l}z" for l in letters) + ",z->" + letters
    return np.einsum(spec, *factors, w, optimize=True)


def add_noise(rng, Y: np.ndarray, snr_db: Optional[float]) -> np.ndarray:
    if snr_db is None:
        return Y
    sigma = 10.0 ** (-snr_db / 20.0) * np.linalg.norm(Y) / math.sqrt(Y.size)
    return Y + sigma * rng.standard_normal(Y.shape)


def cast_like(Y: np.ndarray, dtype: str) -> np.ndarray:
    """Round Y to the storage dtype and return the float64 values that the
    stored tensor represents ("f64", "f32", "bf16", round to nearest even, or
    "bf16x2": the float32 value as hi + lo, hi = bf16(y), lo = bf16(y - hi))."""
    if dtype == "f64":
        return np.asarray(Y, dtype=np.float64)
    if dtype == "f32":
        return np.asarray(Y, dtype=np.float32).astype(np.float64)
    if dtype in ("bf16", "bf16x2"):
        import torch
        t = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32))
        hi = t.to(torch.bfloat16)
        if dtype == "bf16":
            return hi.to(torch.float64).numpy()
        lo = (t - hi.to(torch.float32)).to(torch.bfloat16)
        return (hi.to(torch.float64) + lo.to(torch.float64)).numpy()
    raise ValueError(dtype)


@dataclasses.dataclass
class Problem:
    """One seeded CP problem: tensor values as float64 (already rounded to
    the storage dtype), the true factors and an initial guess."""
    Y: np.ndarray
    true_factors: List[np.ndarray]
    init: List[np.ndarray]
    R: int
    dtype: str
    mu0: Optional[float]
    name: str

    @property
    def dims(self):
        return tuple(self.Y.shape)


def make_problem(seed: int, dims: Sequence[int], R: int, *, dtype: str = "f64",
                 snr_db: Optional[float] = 30.0, collinearity: Sequence[float] = (),
                 col_scale: Optional[tuple] = None, paper_nu: Optional[float] = None,
                 paper_lambda: bool = False, mu0: Optional[float] = None,
                 init_scale: float = 1.0, name: str = "") -> Problem:
    """General recipe.  ``collinearity[n]`` (if given and > 0) makes mode n's
    columns collinear with expected cosine c; ``paper_nu`` uses Eq. (modify_1)
    in every mode instead; ``col_scale=(lo, hi)`` rescales every factor's
    columns log-uniformly; the initial factors are iid N(0, init_scale^2)."""
    rng = rng_for(seed)
    N = len(dims)
    factors = []
    for n, I in enumerate(dims):
        if paper_nu is not None:
            A = paper_collinear(rng, I, R, paper_nu)
        elif n < len(collinearity) and collinearity[n] > 0:
            A = collinear_columns(rng, I, R, collinearity[n])
        else:
            A = rng.standard_normal((I, R))
        if col_scale is not None:
            A = log_uniform_column_scale(rng, A, *col_scale)
        factors.append(A)
    weights = paper_magnitudes(R, N, paper_nu) if (paper_lambda and paper_nu) else None
    Y = tensor_from_factors(factors, weights)
    Y = add_noise(rng, Y, snr_db)
    Y = cast_like(Y, dtype)
    init = [init_scale * rng.standard_normal((I, R)) for I in dims]
    return Problem(Y=np.asfortranarray(Y), true_factors=factors, init=init, R=R,
                   dtype=dtype, mu0=mu0, name=name)


# ---------------------------------------------------------------------------
# The five workload recipes.  Sizes, ranks, noise and collinearity follow the
# benchmark configurations; "small" variants keep the same structure at sizes
# the oracle finishes in seconds.
# ---------------------------------------------------------------------------

def config1(seed: int = 0) -> Problem:
    """20x20x20, R=5, float64, Gaussian factors, SNR 30 dB, mu0 = 1."""
    return make_problem(seed, (20, 20, 20), 5, dtype="f64", snr_db=30.0, mu0=1.0,
                        name="cp3-20^3-R5-f64")


def config2(seed: int = 0, dims=(200, 200, 200), dtype: str = "f64") -> Problem:
    """200^3, R=20, mode-1 collinearity 0.95, modes 2-3 0.81, SNR 40 dB."""
    return make_problem(seed, dims, 20, dtype=dtype, snr_db=40.0,
                        collinearity=(0.95, 0.81, 0.81),
                        name=f"cp3-{dims[0]}^3-R20-collinear-{dtype}")


def config3(seed: int = 0, dims=(60, 60, 60, 60), dtype: str = "bf16") -> Problem:
    """60^4, R=15, column norms log-uniform over [1e-2, 1e2], SNR 30 dB."""
    return make_problem(seed, dims, 15, dtype=dtype, snr_db=30.0,
                        col_scale=(1e-2, 1e2),
                        name=f"cp4-{dims[0]}^4-R15-scaled-{dtype}")


def config4_specs(seed: int = 0, count: int = 512):
    """Batch of independent N=3 problems: I_n ~ U{10..64}, R ~ U{3..12}."""
    rng = rng_for(seed)
    specs = []
    for i in range(count):
        dims = tuple(int(v) for v in rng.integers(10, 65, size=3))
        R = int(rng.integers(3, 13))
        specs.append((seed * 100003 + i + 1, dims, R))
    return specs


def config4_problem(spec, dtype: str = "f32") -> Problem:
    s, dims, R = spec
    return make_problem(s, dims, R, dtype=dtype, snr_db=30.0, collinearity=(0.8,),
                        name=f"batch-{dims}-R{R}")


def config5_requests(seed: int = 0, rate: float = 200.0, seconds: float = 60.0):
    """Poisson arrivals: 70% 32^3 R=5, 25% 128^3 R=16, 5% 400^3 R=30;
    per-request mode-1 collinearity ~ U[0, 0.95]."""
    rng = rng_for(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        u = rng.uniform()
        if u < 0.70:
            dims, R = (32, 32, 32), 5
        elif u < 0.95:
            dims, R = (128, 128, 128), 16
        else:
            dims, R = (400, 400, 400), 30
        c = float(rng.uniform(0.0, 0.95))
        out.append((t, int(rng.integers(0, 2**31 - 1)), dims, R, c))
    return out


def make_complex_problem(seed: int, dims: Sequence[int], R: int, *, snr_db: Optional[float] = 30.0,
                         collinearity: Sequence[float] = (), init_scale: float = 1.0) -> Problem:
    """Complex-valued recipe (Sec. 6, complex tensors: factors with random
    real and imaginary parts): A^(n) = X + i Y with X, Y iid N(0, 1/2) (or
    collinear columns built the same way from complex Gaussian vectors),
    Y = sum of outer products + complex Gaussian noise with E|noise|^2 =
    sigma^2 at the requested SNR (sigma from ||Y||_F as for real tensors);
    complex N(0, 1/2) + i N(0, 1/2) initial factors."""
    rng = rng_for(seed)
    N = len(dims)
    factors = []
    for n, I in enumerate(dims):
        Z = (rng.standard_normal((I, R)) + 1j * rng.standard_normal((I, R))) / math.sqrt(2.0)
        if n < len(collinearity) and collinearity[n] > 0:
            c = collinearity[n]
            b = (rng.standard_normal((I, 1)) + 1j * rng.standard_normal((I, 1))) / math.sqrt(2.0)
            Z = math.sqrt(c) * b + math.sqrt(1.0 - c) * Z
        factors.append(Z)
    letters = string.ascii_lowercase[:N]
    spec = ",".join(f"{l}z" for l in letters) + "->" + letters
    Y = np.einsum(spec, *factors, optimize=True)
    if snr_db is not None:
        sigma = 10.0 ** (-snr_db / 20.0) * np.linalg.norm(Y) / math.sqrt(Y.size)
        Y = Y + sigma * (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)) / math.sqrt(2.0)
    init = [init_scale * (rng.standard_normal((I, R)) + 1j * rng.standard_normal((I, R))) / math.sqrt(2.0)
            for I in dims]
    return Problem(Y=np.asfortranarray(Y), true_factors=factors, init=init, R=R, dtype="c128", mu0=None,
                   name=f"complex-{dims}-R{R}")
