"""The delta-encoding study of the paper's random-graph figure (Sec. III-A,
"Delta-encoding", Fig. 3): for Erdos-Renyi, Watts-Strogatz and Barabasi-Albert
graphs with average degree about 5, 10 and 20, the empirical entropy of the
adjacency matrix's column indices drops when each row's indices are stored as
the first index followed by differences.  The figure plots H(deltas) /
H(indices) over growing node counts; this test computes the same ratio (median
of three seeds) with the oracle's entropy (Eq. 1) and checks the figure's
claim that it is below 1 for every model and degree.  CPU only."""
import numpy as np
import pytest

import oracle as O

nx = pytest.importorskip("networkx")


def _graph(model, n, degree, seed):
    if model == "erdos_renyi":
        return nx.fast_gnp_random_graph(n, degree / (n - 1), seed=seed)
    if model == "watts_strogatz":
        return nx.watts_strogatz_graph(n, degree, 0.1, seed=seed)  # odd degree: degree - 1 ring neighbours
    return nx.barabasi_albert_graph(n, max(1, round(degree / 2)), seed=seed)


def _csr(G):
    n = G.number_of_nodes()
    rows = [sorted(G.neighbors(i)) for i in range(n)]
    lens = np.array([len(r) for r in rows], np.int64)
    cols = np.concatenate([np.array(r, np.int64) for r in rows if r]) if lens.sum() else np.zeros(0, np.int64)
    return lens, cols


def _entropy(symbols):
    _, counts = np.unique(symbols, return_counts=True)
    return O.entropy(counts.astype(np.uint64))


def relative_entropy(model, n, degree, seeds=(0, 1, 2)):
    """H(per-row delta-encoded indices) / H(indices), median over seeds."""
    out = []
    for s in seeds:
        lens, cols = _csr(_graph(model, n, degree, s))
        starts = np.r_[0, np.cumsum(lens)[:-1]]
        deltas = cols.copy()
        deltas[1:] -= cols[:-1]
        first = starts[lens > 0]
        deltas[first] = cols[first]  # each row starts with its absolute index
        out.append(_entropy(deltas) / _entropy(cols))
    return float(np.median(out))


@pytest.mark.parametrize("model", ["erdos_renyi", "watts_strogatz", "barabasi_albert"])
@pytest.mark.parametrize("degree", [5, 10, 20])
def test_delta_encoding_lowers_index_entropy(model, degree):
    ratios = [relative_entropy(model, n, degree) for n in (1000, 4000)]
    assert all(r < 1.0 for r in ratios), ratios


def test_delta_entropy_of_a_band_is_small():
    """A control with a known answer: on a ring lattice (every node joined to
    its 10 nearest neighbours, no rewiring) the deltas of interior rows are
    the same few values, so their entropy is a small fraction of the indices'."""
    assert relative_entropy("watts_strogatz", 4000, 10, seeds=(0,)) < 1.0
    G = nx.watts_strogatz_graph(4000, 10, 0.0, seed=0)
    lens, cols = _csr(G)
    starts = np.r_[0, np.cumsum(lens)[:-1]]
    deltas = cols.copy()
    deltas[1:] -= cols[:-1]
    deltas[starts] = cols[starts]
    assert _entropy(deltas) / _entropy(cols) < 0.5
