"""CPU oracle (test infrastructure only; see oracle.py for the definition)."""
from .oracle import (norm2, dot_seq, cosine_scores, knn, knn_segments,  # noqa: F401
                     recommend, gather, exact_integer_inputs, standardize_stats, standardize,
                     metric_distances, knn_metric, METRICS)
