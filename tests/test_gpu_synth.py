"""The device twin of the genotype generator (synth/synth_gpu.cu) writes the
same packed matrix as the C generator, byte for byte: discrete and admixed
populations, the two-population +-delta model, the null model, the Beta base
frequencies, missing rates from 0 to 1, ragged n and the 10,000 x 100,000
workload in full."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SPECS = [
    synth.GenoSpec(n=1, m=1, seed=3),
    synth.GenoSpec(n=37, m=301, n_pops=2, pm_delta=True, delta_sd=0.05, miss_rate=0.1, seed=5),
    synth.GenoSpec(n=1000, m=777, n_pops=5, admixture=True, miss_rate=0.02, seed=7),
    synth.GenoSpec(n=4099, m=513, n_pops=20, admixture=True, base=("beta", 0.5, 2.0, 0.01, 0.5), miss_rate=0.01,
                   seed=11),
    synth.GenoSpec(n=2051, m=300, n_pops=3, admixture=False, miss_rate=0.0, seed=13),
    synth.GenoSpec(n=515, m=64, n_pops=1, miss_rate=1.0, seed=17),
    synth.null_variant(synth.GenoSpec(n=3001, m=1000, n_pops=5, admixture=True, miss_rate=0.02, seed=19)),
]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.n}x{s.m}-S{s.n_pops}")
def test_device_generator_matches_host(spec):
    host = synth.genotypes(spec).packed
    dev, f, q = synth.genotypes_device(spec)
    assert np.array_equal(dev.cpu().numpy(), host)


def test_device_generator_full_benchmark_workload():
    spec = synth.CONFIGS["fp32_pro_10k_x_100k"].geno
    host = synth.genotypes(spec).packed
    dev, _, _ = synth.genotypes_device(spec)
    assert np.array_equal(dev.cpu().numpy(), host)
