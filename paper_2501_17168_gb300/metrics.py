"""Throughput metric of Sec. V-C.

GPops/s = G * P * S * D / T (Langdon's definition as used by the paper): G
generations, P trees, S the mean node count (leaves included), D data points,
T seconds.  One fitness evaluation of a population is G = 1, so the metric of
this library, node-point evaluations per second, is sum_p len_p * D / T.
"""


def gpops(G: float, P: float, S: float, D: float, T: float) -> float:
    return G * P * S * D / T


def node_point_evals(lengths, D: int) -> float:
    """Node-point evaluations of one pass: sum of tree lengths times points."""
    return float(sum(int(x) for x in lengths)) * float(D)
