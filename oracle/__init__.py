"""FP64 CPU oracle of the fused image-kernel chain.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package. The library's product path
never touches it, and it shares no code with the CUDA path.

`chain` wraps the C oracle (kf_oracle.c, compiled with gcc on first use);
`pchain` is the paper's own chain (Table II / Table IV: gray, IIR, Gaussian, gradient,
threshold, then Kalman) in numpy;
`partition` restates the paper's traffic model and enumerates partitions by brute
force (Sec. VI, Fig. 5, Sec. VI-D);
`stbox` is a spatio-temporal fusable set (temporal binomial, Gaussian, gradient,
threshold) on exact integers and the box traffic behind Eq. 3 - Eq. 6;
`dag` defines the random-DAG stages and `mlp` the cost model's network and gradient;
`dag_plan` restates plans of kernel DAGs that recompute nodes instead of storing them
(members, stores, halos, traffic, on-chip bytes) and finds the cheapest by brute force.
"""
