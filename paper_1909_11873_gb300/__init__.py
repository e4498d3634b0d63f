"""Batched TaylorF2 Gaussian-noise log-likelihood and nested-sampling replacement on GB300 (sm_103a)."""
