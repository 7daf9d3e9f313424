"""Host-side logic on the CPU: the synthetic workload recipes, the
time-to-permeability extraction and the warm-start domain draws.  None of it
needs a GPU or the oracle."""
import numpy as np
import pytest

from paper_1609_09685_gb300 import sharding, workloads


def test_tau_sweep_is_the_papers_grid():
    """Sec. 2: three resolutions at the stated porosities, tau - 1/2 from 0.01
    to 1.5, each (resolution, tau) pair a domain; the pressure difference stays
    in the Stokes regime (at most 1e-3)."""
    wl = workloads.tau_sweep()
    assert len(wl.domains) == 24
    sizes = sorted({(d.nx, d.ny, d.porosity) for d in wl.domains})
    assert sizes == [(400, 200, 0.7394), (800, 400, 0.7532), (1200, 600, 0.7578)]
    taus = sorted({round(d.tau - 0.5, 6) for d in wl.domains})
    assert taus == [0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0, 1.5]
    for d in wl.domains:
        assert 0 < d.drho <= 1e-3
        assert d.drho == pytest.approx(min(1e-3, 1e-4 * (d.tau - 0.5) / 3.0 * (d.nx - 1)))


def test_batch128_ranges_and_determinism():
    a, b = workloads.batch128(), workloads.batch128()
    assert [(d.nx, d.seed, d.tau) for d in a.domains] == [(d.nx, d.seed, d.tau) for d in b.domains]
    assert len(a.domains) == 128
    for d in a.domains:
        assert 200 <= d.nx <= 1200 and d.nx % 2 == 0 and d.ny == d.nx // 2
        assert 0.6 <= d.porosity <= 0.8 and 0.51 <= d.tau <= 1.5
    assert len({d.seed for d in a.domains}) == 128


def test_d3q19_workload():
    wl = workloads.d3q19_256()
    assert [d.tau for d in wl.domains] == [0.52, 0.6, 0.8, 1.0]
    for d in wl.domains:
        assert (d.nx, d.ny, d.nz, d.porosity) == (256, 128, 128, 0.70)


def test_time_to_k_takes_the_last_entry_into_the_band():
    from paper_1609_09685_gb300.warmstart import time_to_k
    t = np.arange(6, dtype=float)
    k = np.array([2.0, 1.5, 1.00005, 0.99, 1.00002, 1.0])
    # the last value outside 1e-4 of the final k is index 3, so the answer is t[4]
    assert time_to_k(t, k, 1e-4) == (4.0, 4)
    assert time_to_k(t, np.ones(6), 1e-4) == (0.0, 0)
    assert time_to_k(t, np.array([]), 1e-4) == (None, None)
    # against a reference k (the oracle's): the band moves with it
    assert time_to_k(t, k, 1e-4, k_ref=1.00003) == (4.0, 4)
    assert time_to_k(t, k, 2e-5, k_ref=1.00003) == (None, None)  # the last k is 3e-5 off
    assert time_to_k(t, k, 1e-4, k_ref=0.99) == (None, None)


def test_warm_start_domain_draws_are_seeded_and_in_range():
    from paper_1609_09685_gb300 import warmstart
    a = warmstart.make_domains(50, (256, 512), seed0=1_000_000, master_seed=12)
    b = warmstart.make_domains(50, (256, 512), seed0=1_000_000, master_seed=12)
    assert a == b
    assert [s for s, _, _ in a] == list(range(1_000_000, 1_000_050))
    for _, phi, tau in a:
        assert 0.6 <= phi <= 0.8 and 0.51 <= tau <= 1.5
    # training and evaluation seeds are disjoint
    train = warmstart.make_domains(512, (256, 512), seed0=0, master_seed=11)
    assert not ({s for s, _, _ in train} & {s for s, _, _ in a})


def test_domain_cost_grows_with_size_and_tau():
    c = sharding.domain_cost
    assert c((200, 400), 0.8) > c((100, 200), 0.8)
    assert c((100, 200), 1.4) > c((100, 200), 0.6)
    assert c((4, 8, 16), 0.8) == pytest.approx(4 * 8 * 16 * 16 * (1 + 2 * 0.3))
