"""CPU oracle for the semi-naive TC / SG fixpoints and triangle counting (test
infrastructure only).

Only tests/, the smoke check and the benchmark's CPU-baseline leg import this
package.  The product path never does.  See wg_oracle.cpp for what is computed
and which passage of the paper each step follows.
"""
from .oracle import (build, digest_keys, oracle_sg, oracle_tc, oracle_tc_reach,  # noqa: F401
                     oracle_tc_rows, oracle_triangles, OracleResult)
