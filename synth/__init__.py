"""Seeded synthetic inputs: packed genotype matrices, start vectors and weights.

This module draws random inputs only and holds none of the PCA method's
arithmetic, so the CPU oracle and the CUDA library both consume its output.
The C source (``synth.c``) is compiled on first use with gcc into
``synth/_build/libsynth.so``.

The workloads (``CONFIGS``) are GWAS-cohort-shaped stand-ins; the paper's own
experiments use a dense synthetic matrix (Algorithm 1, section 2), and no real
genotype dataset is needed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libsynth.so")
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


_LIB_GPU = None


def build_gpu(force: bool = False) -> str:
    """Compile synth_gpu.cu (the device twin of synth_pack) with nvcc for
    sm_103a, FP contraction off, into a shared library; return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libsynth_gpu.so")
    src = os.path.join(_HERE, "synth_gpu.cu")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        nvcc = os.environ.get("NVCC", "nvcc")
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false",
                               "-Xcompiler", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def _lib_gpu():
    global _LIB_GPU
    with _LOCK:
        if _LIB_GPU is None:
            lib = ctypes.CDLL(build_gpu())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.synth_pack_gpu.argtypes = [i64, i64, i64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                                           vp, vp, vp, vp, vp, vp]
            lib.synth_pack_gpu.restype = ctypes.c_int
            _LIB_GPU = lib
    return _LIB_GPU


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("n_pops", ctypes.c_int32), ("admixture", ctypes.c_int32),
                ("base_beta", ctypes.c_int32), ("pm_delta", ctypes.c_int32),
                ("base_lo", ctypes.c_double), ("base_hi", ctypes.c_double),
                ("beta_a", ctypes.c_double), ("beta_b", ctypes.c_double),
                ("delta_sd", ctypes.c_double), ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double),
                ("dirichlet_alpha", ctypes.c_double), ("miss_rate", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.synth_philox_block.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.synth_population.argtypes = [P(_Params), ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_population.restype = ctypes.c_int
            lib.synth_pack.argtypes = [P(_Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_pack.restype = ctypes.c_int
            lib.synth_normal_vec.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p]
            lib.synth_uniform_vec.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
            lib.synth_paper_model.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_paper_model.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def padded_stride(n: int) -> int:
    """Row bytes for n samples: ceil(n/4) rounded up to a multiple of 16."""
    return ((n + 3) // 4 + 15) // 16 * 16


@dataclass(frozen=True)
class GenoSpec:
    """Parameters of the genotype model (see synth.c for the model)."""
    n: int
    m: int
    n_pops: int = 1
    admixture: bool = False
    base: tuple = ("uniform", 0.05, 0.5)   # ("uniform", lo, hi) or ("beta", a, b, lo, hi)
    pm_delta: bool = False
    delta_sd: float = 0.05
    f_clip: tuple = (0.01, 0.99)
    dirichlet_alpha: float = 0.5
    miss_rate: float = 0.01
    seed: int = 1

    @property
    def stride(self) -> int:
        return padded_stride(self.n)

    def _params(self) -> _Params:
        p = _Params()
        p.n, p.m, p.stride = self.n, self.m, self.stride
        p.n_pops, p.admixture, p.pm_delta = self.n_pops, int(self.admixture), int(self.pm_delta)
        if self.base[0] == "beta":
            p.base_beta = 1
            p.beta_a, p.beta_b, p.base_lo, p.base_hi = self.base[1:5]
        else:
            p.base_beta = 0
            p.base_lo, p.base_hi = self.base[1:3]
        p.delta_sd = self.delta_sd
        p.f_lo, p.f_hi = self.f_clip
        p.dirichlet_alpha = self.dirichlet_alpha
        p.miss_rate = self.miss_rate
        p.seed = self.seed
        return p


@dataclass
class Genotypes:
    spec: GenoSpec
    packed: np.ndarray      # uint8 [m, stride]
    f: np.ndarray           # float64 [S, m] population allele frequencies
    q: np.ndarray           # float64 [n, S] ancestry proportions

    @property
    def n(self):
        return self.spec.n

    @property
    def m(self):
        return self.spec.m

    @property
    def stride(self):
        return self.spec.stride


def genotypes(spec: GenoSpec, out: np.ndarray | None = None) -> Genotypes:
    """Draw a packed genotype matrix for ``spec`` (deterministic in spec.seed)."""
    lib = _lib()
    p = spec._params()
    f = np.empty((spec.n_pops, spec.m), dtype=np.float64)
    q = np.empty((spec.n, spec.n_pops), dtype=np.float64)
    if lib.synth_population(ctypes.byref(p), f.ctypes.data, q.ctypes.data) != 0:
        raise ValueError("bad genotype spec")
    if out is None:
        out = np.empty((spec.m, spec.stride), dtype=np.uint8)
    assert out.shape == (spec.m, spec.stride) and out.dtype == np.uint8 and out.flags.c_contiguous
    if lib.synth_pack(ctypes.byref(p), f.ctypes.data, q.ctypes.data, out.ctypes.data) != 0:
        raise ValueError("bad genotype spec")
    return Genotypes(spec, out, f, q)


@dataclass(frozen=True)
class ModelSpec:
    """The paper's synthetic genotype model (section 2, Algorithm 1): m markers
    by n patients, r admixture sub-blocks, nsignal_frac * m * n signal draws and
    round(rkins * m) duplicated marker rows (see synth.c)."""
    n: int
    m: int
    r: int = 10
    nsignal_frac: float = 1.0
    rkins: float = 0.017
    seed: int = 0x5EED0006

    @property
    def stride(self) -> int:
        return padded_stride(self.n)


# The matrix size and parameters of the paper's Fig. empirical-spectrum and
# Table 3 (41,505 markers x 81,700 patients, r = 10, nsignal = mn, rkins = 0.017).
PAPER_MODEL = ModelSpec(n=81_700, m=41_505)


def paper_model(spec: ModelSpec, out: np.ndarray | None = None) -> Genotypes:
    """Draw the packed matrix of the paper's model (deterministic in spec.seed)."""
    if out is None:
        out = np.empty((spec.m, spec.stride), dtype=np.uint8)
    assert out.shape == (spec.m, spec.stride) and out.dtype == np.uint8 and out.flags.c_contiguous
    rc = _lib().synth_paper_model(spec.n, spec.m, spec.stride, spec.r, spec.nsignal_frac * spec.m * spec.n,
                                  spec.rkins, spec.seed, out.ctypes.data)
    if rc != 0:
        raise ValueError("bad model spec")
    return Genotypes(spec, out, np.zeros((0, spec.m)), np.zeros((spec.n, 0)))


def genotypes_device(spec: GenoSpec, device="cuda"):
    """The packed matrix of ``genotypes(spec)``, byte for byte, drawn on a CUDA
    device (synth_gpu.cu): the per-SNP and per-sample parameters f and q come
    from the same C code on the host, the per-entry draws from the device.
    Returns (packed uint8 tensor [m, stride] on the device, f, q)."""
    import math

    import torch
    lib = _lib()
    p = spec._params()
    f = np.empty((spec.n_pops, spec.m), dtype=np.float64)
    q = np.empty((spec.n, spec.n_pops), dtype=np.float64)
    if lib.synth_population(ctypes.byref(p), f.ctypes.data, q.ctypes.data) != 0:
        raise ValueError("bad genotype spec")
    dev = torch.device(device)
    q64 = torch.from_numpy(q).to(dev)
    f64 = torch.from_numpy(f).to(dev)
    q32 = torch.from_numpy(q.astype(np.float32)).to(dev)
    f32 = torch.from_numpy(f.astype(np.float32)).to(dev)
    out = torch.empty((spec.m, spec.stride), dtype=torch.uint8, device=dev)
    # (double) r < miss_rate * 2^32  <=>  r < ceil(miss_rate * 2^32) for an integer r
    miss_int = min(int(math.ceil(spec.miss_rate * 4294967296.0)), 1 << 32)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream().cuda_stream
        rc = _lib_gpu().synth_pack_gpu(spec.n, spec.m, spec.stride, spec.n_pops, spec.seed, miss_int,
                                       q64.data_ptr(), f64.data_ptr(), q32.data_ptr(), f32.data_ptr(),
                                       out.data_ptr(), stream)
        if rc != 0:
            raise RuntimeError(f"synth_pack_gpu failed ({rc})")
        torch.cuda.current_stream().synchronize()
    return out, f, q


def normal_vec(seed: int, stream: int, length: int) -> np.ndarray:
    out = np.empty(length, dtype=np.float64)
    _lib().synth_normal_vec(seed, stream, length, out.ctypes.data)
    return out


def uniform_vec(seed: int, stream: int, length: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(length, dtype=np.float64)
    _lib().synth_uniform_vec(seed, stream, length, lo, hi, out.ctypes.data)
    return out


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (for known-answer tests)."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _lib().synth_philox_block(c, k, o)
    return tuple(int(x) for x in o)


@dataclass(frozen=True)
class Workload:
    """A genotype matrix plus the solver settings it is measured with."""
    name: str
    geno: GenoSpec
    k: int
    ell: int
    reorth: str
    precision: str
    tol: float
    extra: dict = field(default_factory=dict)


# Five GWAS-shaped workloads.  Sizes, population structure, missingness and
# solver settings follow the hot-path scope of this library; the small one is
# cheap enough for the CPU oracle to solve in seconds.
CONFIGS = {
    "fp64_full_1k_x_10k": Workload(
        "fp64_full_1k_x_10k",
        GenoSpec(n=1000, m=10_000, n_pops=2, admixture=False, pm_delta=True, delta_sd=0.05,
                 f_clip=(0.01, 0.99), miss_rate=0.01, seed=0x5EED0001),
        k=10, ell=30, reorth="full", precision="fp64", tol=1e-10),
    "fp32_pro_10k_x_100k": Workload(
        "fp32_pro_10k_x_100k",
        GenoSpec(n=10_000, m=100_000, n_pops=5, admixture=True, dirichlet_alpha=0.5,
                 delta_sd=0.05, miss_rate=0.02, seed=0x5EED0002),
        k=20, ell=50, reorth="partial", precision="fp32", tol=1e-6),
    "block_50k_x_500k": Workload(
        "block_50k_x_500k",
        GenoSpec(n=50_000, m=500_000, n_pops=10, admixture=True, miss_rate=0.01, seed=0x5EED0003),
        k=20, ell=128, reorth="full", precision="block", tol=1e-6, extra={"block": 16, "k_keep": 48}),
    "grad_20k_x_200k": Workload(
        "grad_20k_x_200k",
        GenoSpec(n=20_000, m=200_000, n_pops=5, admixture=True, miss_rate=0.0, seed=0x5EED0004),
        k=10, ell=40, reorth="full", precision="fp32", tol=1e-8, extra={"weights": (0.5, 1.5)}),
    "large_200k_x_1m": Workload(
        "large_200k_x_1m",
        GenoSpec(n=200_000, m=1_000_000, n_pops=20, admixture=True,
                 base=("beta", 0.5, 2.0, 0.01, 0.5), miss_rate=0.01, seed=0x5EED0005),
        k=20, ell=50, reorth="dgks", precision="fp32", tol=1e-6,
        extra={"block": 16, "block_ell": 128, "k_keep": 48, "grad": "w"}),
}


def null_variant(spec: GenoSpec) -> GenoSpec:
    """The same shape with no population structure (f_kj = p_j)."""
    return replace(spec, delta_sd=0.0, n_pops=1, admixture=False, pm_delta=False)
