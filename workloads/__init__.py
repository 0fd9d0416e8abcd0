"""Seeded synthetic inputs shared by the CUDA path's tests/benchmarks and the
CPU oracle.  Holds geometry and boundary-data generation only -- none of the
time-spectral GLS arithmetic."""
