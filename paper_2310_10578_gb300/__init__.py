"""GB300-native creeping-wave (smooth-surface UTD) field evaluator."""
