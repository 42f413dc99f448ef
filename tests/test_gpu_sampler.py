"""Chain-rule threshold-detector sampling (tor_sample) against the oracle.

The probability of clicks on S and none on the other modes of the first j
modes is Tor(O^(j)_S) / sqrt(det Sigma_[j]) with O^(j) = I - Sigma_[j]^{-1}
(Sec. 1, Eq. A applied to the marginal state).  Here those probabilities come
from the binary128 oracle on O^(j) built by the seeded generator, and the
sampler is checked three ways: the probability it reports for each drawn
pattern, every one of its click decisions replayed with the exact conditional
probabilities, and the frequencies of the patterns it draws.
"""
import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2109_04528_gb300 import build
    build.build()
    c = binding.Context(device=0)
    yield c
    c.close()


class Exact:
    """P(clicks S, no click on the other modes of 0..j-1) from the oracle."""

    def __init__(self, oracle_mod, sigma):
        self.o, self.sigma, self.n = oracle_mod, sigma, sigma.shape[0] // 2
        self.cache, self.scale = {}, {}

    def prefix(self, j):
        if j not in self.scale:
            idx = np.concatenate([np.arange(j), self.n + np.arange(j)])
            sj = self.sigma[np.ix_(idx, idx)]
            self.scale[j] = (inputs.sampling_matrix(sj), 1.0 / np.sqrt(np.linalg.det(sj).real))
        return self.scale[j]

    def __call__(self, j, S):
        key = (j, tuple(S))
        if key not in self.cache:
            Oj, sc = self.prefix(j)
            if S:
                r = self.o.tor_brute(inputs.submatrix(Oj, list(S)))
                self.cache[key] = ((r.hi + r.lo) * sc, r.abs_sum * sc)
            else:
                self.cache[key] = (sc, sc)
        return self.cache[key]


def clicks(row):
    return [j for j, c in enumerate(row) if c]


def test_probabilities_and_decisions(ctx, oracle_mod):
    inst = inputs.lossy_squeezed(8, 2021, (0.5, 1.2), 0.5)
    u = inputs.rng_for(7).uniform(0.0, 1.0, size=(300, 8))
    with binding.Session(ctx, inst.sigma) as sess:
        pat, prob, dev = binding.tor_sample(ctx, sess, u)
    ex = Exact(oracle_mod, inst.sigma)
    assert dev <= 1e-10
    close = 0
    for i in range(len(u)):
        # every decision, replayed with the exact conditionals
        S = []
        for j in range(8):
            p0, _ = ex(j + 1, S)
            p1, _ = ex(j + 1, S + [j])
            c = p1 / (p0 + p1)
            if abs(u[i, j] - c) < 1e-9:
                close += 1
                S = clicks(pat[i][: j + 1])
                continue
            assert pat[i, j] == (u[i, j] < c), (i, j)
            if pat[i, j]:
                S = S + [j]
        # the reported probability of the drawn pattern
        want, absum = ex(8, clicks(pat[i]))
        assert abs(prob[i] - want) <= 1e-10 * absum, (i, prob[i], want)
    assert close <= 2


def test_pattern_frequencies(ctx, oracle_mod):
    pytest.importorskip("scipy")
    from scipy.stats import chi2
    inst = inputs.lossy_squeezed(10, 77, (0.5, 1.2), 0.4)
    n_modes, count = 4, 6000
    u = inputs.rng_for(11).uniform(0.0, 1.0, size=(count, n_modes))
    with binding.Session(ctx, inst.sigma) as sess:
        pat, prob, dev = binding.tor_sample(ctx, sess, u)
    ex = Exact(oracle_mod, inst.sigma)
    exp = np.array([ex(n_modes, [j for j in range(n_modes) if m >> j & 1])[0] for m in range(1 << n_modes)])
    assert abs(exp.sum() - 1.0) <= 1e-12
    codes = (pat.astype(np.int64) << np.arange(n_modes)).sum(axis=1)
    obs = np.bincount(codes, minlength=1 << n_modes)
    assert np.allclose(prob, exp[codes], rtol=1e-9, atol=0)
    keep = exp * count >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum()) * count
    stat = float(((o - e) ** 2 / np.maximum(e, 1e-300)).sum())
    assert chi2.sf(stat, len(o) - 1) > 1e-3, (stat, o, e)


def test_extended_sampler_on_weak_squeezing(oracle_mod):
    # Sec. 5: weak squeezing, cancelling Torontonians: the extended context
    # gives the patterns' probabilities to many digits
    inst = inputs.lossy_squeezed(10, 4256, (0.1, 0.2), 1.0)
    u = inputs.rng_for(5).uniform(0.0, 1.0, size=(40, 10))
    with binding.Context(device=0, flags=binding.TOR_EXTENDED) as cx, binding.Session(cx, inst.sigma) as sess:
        pat, prob, dev = binding.tor_sample(cx, sess, u)
    ex = Exact(oracle_mod, inst.sigma)
    assert dev <= 1e-12
    for i in range(len(u)):
        want, _ = ex(10, clicks(pat[i]))
        assert abs(prob[i] - want) <= 1e-8 * abs(want), (i, prob[i], want)


def test_arguments(ctx):
    inst = inputs.lossy_squeezed(5, 3, (0.5, 1.2), 0.5)
    with binding.Session(ctx, inst.sigma) as sess:
        pat, prob, dev = binding.tor_sample(ctx, sess, np.zeros((0, 5)))
        assert pat.shape == (0, 5)
        with pytest.raises(binding.TorError) as e:
            binding.tor_sample(ctx, sess, np.full((2, 6), 0.5))  # more modes than the state
        assert e.value.status == binding.TOR_EINVAL
        with pytest.raises(binding.TorError) as e:
            binding.tor_sample(ctx, sess, np.full((2, 5), 1.0))  # a uniform outside [0, 1)
        assert e.value.status == binding.TOR_EINVAL
        # all-zero uniforms click wherever the conditional is positive: every mode
        # of a squeezed state
        pat, prob, _ = binding.tor_sample(ctx, sess, np.zeros((1, 5)))
        assert pat.sum() == 5


def test_chunks_shrink_under_a_memory_budget():
    # a budget that holds the fixed scratch and a quarter of what a whole step's 2 x 3000
    # marginals add to it: the steps are split into smaller launches, the draws are the same
    inst = inputs.lossy_squeezed(14, 77, (0.5, 1.2), 0.5)
    u = inputs.rng_for(9).uniform(0.0, 1.0, size=(3000, 14))
    with binding.Context(device=0) as c, binding.Session(c, inst.sigma) as sess:
        want = binding.tor_sample(c, sess, u)
        full = c.memory()[0]
    kmax = min(14, int(want[0].sum(axis=1).max()) + 1)  # the largest continuation S u {j} evaluated
    with binding.Context(device=0) as probe, binding.Session(probe, inst.sigma) as sess:
        # the scratch of the largest marginal and of the largest one-lane-per-unit size (p < 5)
        for k in sorted({kmax, min(kmax, 8)}):
            assert binding.tor_eval_marginal(probe, sess, 14, list(range(k))).status == 0
        fixed = probe.memory()[0]
    assert full > fixed + (4 << 20), (full, fixed)
    budget = fixed + (full - fixed) // 4
    with binding.Context(device=0, mem_budget=budget) as c, binding.Session(c, inst.sigma) as sess:
        got = binding.tor_sample(c, sess, u)
        assert c.memory()[0] <= budget
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])


def test_graph_context_draws_the_same():
    # a context with TOR_GRAPHS draws the same patterns (its sampling steps run uncaptured:
    # each has a new shape) and keeps its graph cache for the calls that repeat
    inst = inputs.lossy_squeezed(12, 61, (0.5, 1.2), 0.5)
    u = inputs.rng_for(13).uniform(0.0, 1.0, size=(200, 12))
    with binding.Context(device=0) as c, binding.Session(c, inst.sigma) as sess:
        want = binding.tor_sample(c, sess, u)
    with binding.Context(device=0, flags=binding.TOR_GRAPHS) as c, binding.Session(c, inst.sigma) as sess:
        got = binding.tor_sample(c, sess, u)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
