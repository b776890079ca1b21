"""CPU oracle (test infrastructure only): a plain FP64 restatement of the
geometric adaptive smoothed aggregation method.  Only tests, the smoke check
and the benchmark's CPU-baseline leg may import it."""
