"""Seeded synthetic inputs: genotypes and phenotypes.

This module only draws random inputs.  It holds none of the method's
arithmetic, so both the CUDA path's tests/benchmark and the CPU oracle's tests
can use it without sharing any computation.

Recipe (the paper's UK BioBank and msprime cohorts are not available here;
these draws stand in for them with the same value range and shapes):

* allele frequency per SNP: ``p_j ~ U(0.05, 0.5)``, drawn on the CPU from
  ``torch.Generator().manual_seed(seed)`` so it does not depend on the device;
* genotype ``g_ij = [u1_ij < p_j] + [u2_ij < p_j]`` (Binomial(2, p_j)), values
  {0, 1, 2} stored as int8, uniforms drawn on ``device`` from a generator
  seeded with ``seed + 1`` (CPU and CUDA generators give different streams;
  a test that compares two implementations hands both the same tensor);
* phenotype column c: 20 SNP pairs (a, b) drawn without replacement from the
  SNPs, weights ``w ~ N(0, 1)``, noise ``e ~ N(0, 0.5^2)``:
  ``y_ic = sum_t w_ct g_{i,a_t} g_{i,b_t} + e_ic``, accumulated in float64 and
  stored float32;
* held-out rows are further rows of the same genotype stream (same p_j).

Structured cohorts (``structured_problem``; the FP8-dominant regime): the
rows come from ``populations`` subpopulations under the Balding-Nichols
model -- ancestral ``p_j ~ U(0.05, 0.5)`` as above, population ``k`` draws
``p_kj ~ Beta(p_j (1 - F) / F, (1 - p_j) (1 - F) / F)`` (mean ``p_j``,
variance ``F p_j (1 - p_j)``, ``F`` the fixation index) from a numpy
generator seeded with ``seed + 3``; training rows are grouped by population
in equal contiguous blocks, held-out rows likewise; genotypes and phenotypes
then follow the recipe above with each row's own population frequencies.
"""
from __future__ import annotations

import numpy as np
import torch

N_PAIRS = 20
NOISE_SD = 0.5


def allele_freqs(m: int, seed: int) -> torch.Tensor:
    g = torch.Generator().manual_seed(int(seed))
    return 0.05 + 0.45 * torch.rand(m, generator=g, dtype=torch.float64)


def genotypes(n: int, m: int, seed: int, device="cpu", chunk_rows: int = 8192) -> torch.Tensor:
    """n x m int8 genotype matrix, rows = patients, values in {0, 1, 2}."""
    device = torch.device(device)
    p = allele_freqs(m, seed).to(device=device, dtype=torch.float32)
    gen = torch.Generator(device=device).manual_seed(int(seed) + 1)
    out = torch.empty((n, m), dtype=torch.int8, device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        u = torch.rand((r1 - r0, m), generator=gen, device=device, dtype=torch.float32)
        blk = (u < p).to(torch.int8)
        torch.rand((r1 - r0, m), generator=gen, device=device, dtype=torch.float32, out=u)
        blk += (u < p).to(torch.int8)
        out[r0:r1] = blk
        del u, blk
    return out


def phenotypes(g: torch.Tensor, n_pheno: int, seed: int) -> torch.Tensor:
    """n x n_pheno float32 phenotypes from pairwise SNP products plus noise."""
    n, m = g.shape
    gen = torch.Generator().manual_seed(int(seed) + 2)
    cols = []
    for _ in range(n_pheno):
        snps = torch.randperm(m, generator=gen)[: 2 * N_PAIRS]
        w = torch.randn(N_PAIRS, generator=gen, dtype=torch.float64)
        a, b = snps[:N_PAIRS].to(g.device), snps[N_PAIRS:].to(g.device)
        prod = g[:, a].to(torch.float64) * g[:, b].to(torch.float64)
        cols.append(prod @ w.to(g.device))
    y = torch.stack(cols, dim=1)
    noise = torch.randn((n, n_pheno), generator=gen, dtype=torch.float64) * NOISE_SD
    return (y + noise.to(g.device)).to(torch.float32)


def problem(n: int, m: int, n_pheno: int, n_test: int, seed: int, device="cpu"):
    """Training genotypes/phenotypes and held-out genotypes/phenotypes.

    Returns a dict with G (n x m int8), Y (n x P float32), T (n_test x m int8)
    and Yt (n_test x P float32), all on ``device``.
    """
    g_all = genotypes(n + n_test, m, seed, device=device)
    y_all = phenotypes(g_all, n_pheno, seed)
    return {"G": g_all[:n].contiguous(), "Y": y_all[:n].contiguous(),
            "T": g_all[n:].contiguous(), "Yt": y_all[n:].contiguous()}


def population_freqs(m: int, populations: int, fst: float, seed: int) -> torch.Tensor:
    """populations x m allele frequencies under the Balding-Nichols model."""
    p0 = allele_freqs(m, seed).numpy()
    rng = np.random.default_rng(int(seed) + 3)
    shape = (1.0 - fst) / fst
    pk = rng.beta(p0 * shape, (1.0 - p0) * shape, size=(populations, m))
    return torch.from_numpy(pk)


def _population_of(rows: int, populations: int) -> torch.Tensor:
    """Equal contiguous blocks: row r belongs to population r * populations // rows."""
    return torch.arange(rows, dtype=torch.int64) * populations // max(rows, 1)


def structured_genotypes(n: int, m: int, seed: int, pk: torch.Tensor, pop: torch.Tensor, device="cpu",
                         chunk_rows: int = 8192) -> torch.Tensor:
    """n x m int8 genotypes, row r drawn with the frequencies of population pop[r]."""
    device = torch.device(device)
    pkd = pk.to(device=device, dtype=torch.float32)
    popd = pop.to(device)
    gen = torch.Generator(device=device).manual_seed(int(seed) + 1)
    out = torch.empty((n, m), dtype=torch.int8, device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        pr = pkd[popd[r0:r1]]
        u = torch.rand((r1 - r0, m), generator=gen, device=device, dtype=torch.float32)
        blk = (u < pr).to(torch.int8)
        torch.rand((r1 - r0, m), generator=gen, device=device, dtype=torch.float32, out=u)
        blk += (u < pr).to(torch.int8)
        out[r0:r1] = blk
        del u, blk, pr
    return out


def structured_problem(n: int, m: int, n_pheno: int, n_test: int, seed: int, populations: int = 8,
                       fst: float = 0.3, device="cpu"):
    """Training and held-out data of ``populations`` structured cohorts.

    Returns the keys of ``problem`` plus ``pop`` and ``pop_test`` (the
    population index of every training and held-out row)."""
    pk = population_freqs(m, populations, fst, seed)
    pop = _population_of(n, populations)
    pop_t = _population_of(n_test, populations)
    g_all = structured_genotypes(n + n_test, m, seed, pk, torch.cat([pop, pop_t]), device=device)
    y_all = phenotypes(g_all, n_pheno, seed)
    return {"G": g_all[:n].contiguous(), "Y": y_all[:n].contiguous(),
            "T": g_all[n:].contiguous(), "Yt": y_all[n:].contiguous(), "pop": pop, "pop_test": pop_t}


def confounders(n: int, nc: int, seed: int, scale: float = 1.0) -> torch.Tensor:
    """n x nc FP32 real-valued covariates (stand-ins for age, sex, ancestry
    principal components): independent N(0, scale^2) draws from a CPU
    generator seeded with ``seed + 4``."""
    g = torch.Generator().manual_seed(int(seed) + 4)
    return (torch.randn((n, nc), generator=g, dtype=torch.float64) * scale).to(torch.float32)
