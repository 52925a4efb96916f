"""One generation of the tree-based GP loop on the device (Algorithm 1).

Fitness (SR mean squared error, Sec. III-C) -> tournament selection of two
parents per child -> one-point crossover with probability ``p_cross`` ->
subtree mutation with probability ``p_mut`` (Sec. III-B), with the paper's
defaults from the table "Configuration of Genetic Programming" (maximum tree
size 512, tournament size 20, crossover 0.9, mutation 0.1).  Every step runs
in the library's kernels; torch only holds the buffers and draws the random
words.  All buffers are allocated up front, so ``step`` can be captured in a
CUDA graph and replayed once per generation.

The "newly generated subtrees" of subtree mutation come from a pool of random
trees supplied by the caller; mutation replaces a random node of the child by
a whole pool tree chosen at random.
"""
from __future__ import annotations

import torch

from . import _lib, api


def _threshold(p: float) -> int:
    """A child takes part when its 32-bit word is below p * 2^32."""
    return min(int(round(p * 2 ** 32)), 2 ** 32 - 1) if p < 1 else 2 ** 32 - 1


class Generation:
    """Device-resident state of the GP loop for one SR problem.

    ``pop`` is a (type, value, size) tuple of float32 [P, ld] tensors with
    ld >= max_size; it is updated in place by ``step``.  ``pool`` is a
    (type, value, size) tuple of the mutation trees.
    """

    def __init__(self, pop, X, y, pool, max_size: int = 512, tournament_size: int = 20,
                 p_cross: float = 0.9, p_mut: float = 0.1, generator=None):
        self.pop = pop
        self.X, self.y = X, y
        self.pool = pool
        self.max_size = max_size
        self.t = tournament_size
        P, ld = pop[0].shape
        if ld < max_size:
            raise ValueError("population rows must hold max_size nodes")
        self.P, self.ld = P, ld
        dev = X.device
        self.gen = generator
        self.tmp = tuple(torch.empty_like(a) for a in pop)
        self.mse = torch.empty((P, 1), dtype=torch.float64, device=dev)
        self.status = torch.empty(P, dtype=torch.int32, device=dev)
        self.words = torch.empty(2 * P * self.t + 5 * P, dtype=torch.int32, device=dev)
        self.pool_index = torch.empty(P, dtype=torch.int32, device=dev)
        self.rows = torch.arange(P, dtype=torch.int32, device=dev)
        self.winners = torch.empty(2 * P, dtype=torch.int32, device=dev)
        w = self.words
        n_t = 2 * P * self.t
        self.w_tour = w[:n_t].view(2 * P, self.t)
        self.w_k1, self.w_j1, self.w_a1, self.w_k2, self.w_a2 = (
            w[n_t + i * P:n_t + (i + 1) * P] for i in range(5))
        self.thr_cross, self.thr_mut = _threshold(p_cross), _threshold(p_mut)
        self.cross_status = torch.empty(P, dtype=torch.int32, device=dev)
        self.mut_status = torch.empty(P, dtype=torch.int32, device=dev)

    def draw(self):
        """Fresh random words for one generation (torch's device generator)."""
        self.words.random_(-2 ** 31, 2 ** 31, generator=self.gen)
        self.pool_index.random_(0, self.pool[0].shape[0], generator=self.gen)

    def apply(self):
        """Fitness, selection, crossover and mutation with the drawn words;
        returns the fitness of the population it started from."""
        api.tgp_fitness_mse(*self.pop, self.X, self.y, 1, max_len=self.max_size, mse=self.mse,
                            tree_status=self.status)
        api.tgp_tournament_select(self.mse[:, 0], self.w_tour, True, winners=self.winners)
        p1, p2 = self.winners[:self.P], self.winners[self.P:]
        _, self.cross_status = api.tgp_subtree_exchange(
            self.pop, p1, self.w_k1, donor=self.pop, donor_index=p2, donor_node=self.w_j1,
            mode=_lib.PICK_RANDOM, max_size=self.max_size, out_ld=self.ld,
            apply_word=self.w_a1, apply_below=self.thr_cross, old_max_len=self.max_size,
            donor_max_len=self.max_size, out=self.tmp, status=self.cross_status)
        _, self.mut_status = api.tgp_subtree_exchange(
            self.tmp, self.rows, self.w_k2, donor=self.pool, donor_index=self.pool_index,
            donor_node=None, mode=_lib.PICK_RANDOM, max_size=self.max_size, out_ld=self.ld,
            apply_word=self.w_a2, apply_below=self.thr_mut, old_max_len=self.max_size,
            out=self.pop, status=self.mut_status)
        return self.mse

    def step(self):
        self.draw()
        return self.apply()
