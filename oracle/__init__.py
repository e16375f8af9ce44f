"""FP64 CPU oracle of the spectral-quadrature hot path: test infrastructure only (tests/, the
package smoke check and bench.py's CPU-baseline leg).  Never imported by the product path."""
