"""CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
legs may import this package.  The GPU library never imports or links it and
the two share no code.  See oracle/hphi_oracle.c for the definitions and
oracle/spectrum.py for the dynamical correlation function (resolvent,
continued fraction, shifted COCG).
"""
from .oracle import (build, num_threads, Model, binom, enumerate_states, rank_colex, unrank_colex, lin_tables,
                     tridiag_eig, tridiag_vec, sturm_count, dense_matrix, canonical_thermo, bootstrap_tpq,
                     MODELS, KINDS)

__all__ = ["build", "num_threads", "Model", "binom", "enumerate_states", "rank_colex", "unrank_colex", "lin_tables",
           "tridiag_eig", "tridiag_vec", "sturm_count", "dense_matrix", "canonical_thermo", "bootstrap_tpq",
           "MODELS", "KINDS"]
